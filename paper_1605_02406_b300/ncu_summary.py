"""Summaries of Nsight Compute CSV logs of the filter's kernels.

    python -m paper_1605_02406_b300.ncu_summary launches LOG.csv      # markdown table
    python -m paper_1605_02406_b300.ncu_summary traffic LOG.csv OUT.json --steps-from LOG
    python -m paper_1605_02406_b300.ncu_summary kernel RAW.csv ALG_BYTES    # one --set full launch
    python -m paper_1605_02406_b300.ncu_summary first-step LOG.csv    # ncu -s past the autotuner

`launches` reads a `--metrics gpu__time_duration.sum --csv` log (one row per launch) and
prints, per kernel, its launches, total time and share of the total.  `traffic` reads a
`--metrics dram__bytes_read.sum,dram__bytes_write.sum --csv` log and writes the DRAM bytes
per launch of each kernel, tagged with the hash of the CUDA sources they were taken from
(bench.py reports them only while the sources are unchanged).
"""
from __future__ import annotations

import collections
import csv
import hashlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def csrc_hash() -> str:
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1605_02406_b300", "csrc")
    for n in sorted(os.listdir(d)):
        with open(os.path.join(d, n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def rows(path: str) -> list:
    lines = open(path).read().splitlines()
    start = next(k for k, line in enumerate(lines) if line.startswith('"ID"'))
    return list(csv.DictReader(io.StringIO("\n".join(lines[start:]))))


def kernel_name(full: str) -> str:
    """'void k_segsum<0>(dog::KParams, ...)' -> 'k_segsum'; '<unnamed>::k_na_hist(...)' ->
    'k_na_hist'"""
    n = full.split("(")[0].replace("void ", "").replace("<unnamed>::", "").strip()
    return n.split("<")[0].split("::")[-1]


def first_step_after_tuning(names: list) -> int:
    """Index of the first launch of the frames that follow the sort autotuner's trials (each
    trial starts with k_na_hist): the next grid take-over or frame tick; 0 without trials."""
    trials = [i for i, k in enumerate(names) if k == "k_na_hist"]
    if not trials:
        return 0
    return next(i for i in range(trials[-1], len(names)) if names[i] in ("k_take_grid", "k_tick"))


def _durations(path: str) -> list:
    out = []
    for r in rows(path):
        if r["Metric Name"] != "gpu__time_duration.sum":
            continue
        scale = {"ns": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}.get(r["Metric Unit"], 1e-3)
        out.append((kernel_name(r["Kernel Name"]), float(r["Metric Value"].replace(",", "")) * scale))
    return out


def launches(path: str) -> str:
    """Per kernel: launches, total time, share, over the frames after the autotuner's
    trials; the launches before them (initial state, first frame, trials) in one line."""
    d = _durations(path)
    s = first_step_after_tuning([k for k, _ in d])
    n = collections.Counter()
    t = collections.defaultdict(float)
    for k, us in d[s:]:
        n[k] += 1
        t[k] += us
    total = sum(t.values())
    out = ["| kernel | launches | total µs | µs / launch | share |", "|---|---|---|---|---|"]
    for k in sorted(t, key=lambda k: -t[k]):
        out.append(f"| {k} | {n[k]} | {t[k]:.1f} | {t[k] / n[k]:.1f} | {100 * t[k] / total:.1f} % |")
    out.append(f"| **all** | {sum(n.values())} | {total:.1f} | | 100 % |")
    if s:
        out += ["", f"Not in the table: the {s} launches before those frames (initial state, first "
                f"frame, sort autotuning trials), {sum(us for _, us in d[:s]):.1f} µs."]
    return "\n".join(out)


def traffic(path: str) -> dict:
    """DRAM bytes per launch by kernel; sort launches are numbered by their pass (the
    first after k_predict is pass 0)."""
    acc = collections.OrderedDict()
    for r in rows(path):
        m = r["Metric Name"]
        if m not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(r["Metric Unit"], 1)
        key = int(r["ID"])
        if key not in acc:
            acc[key] = [kernel_name(r["Kernel Name"]), 0.0]
        acc[key][1] += float(r["Metric Value"].replace(",", "")) * scale
    per = collections.defaultdict(list)
    sort_pass = None
    for _, (k, v) in sorted(acc.items()):
        k = k.replace("_lidar", "")  # the lidar variants report under the step's kernel names
        if k == "k_predict":
            sort_pass = 0
        elif k in ("k_sort_count", "k_sort_offsets", "k_sort_pass"):
            if sort_pass is None:  # capture began inside the sort: pass unknown
                continue
            k = f"{k}{sort_pass}"
            if k.startswith("k_sort_pass"):
                sort_pass += 1
        per[k].append(v)
    return {k: sum(v) / len(v) for k, v in per.items()}


# metrics of a `--set full` capture worth reading for this memory- and issue-bound code
KERNEL_METRICS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("lts__t_bytes.sum", "L2 bytes"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput % of peak"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % (occupancy)"),
    ("launch__registers_per_thread", "registers / thread"),
    ("launch__block_size", "block size"),
    ("launch__grid_size", "grid size"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("l1tex__t_sectors_pipe_lsu_mem_global_op_ld.sum", "global load sectors"),
    ("l1tex__t_requests_pipe_lsu_mem_global_op_ld.sum", "global load requests"),
    ("l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", "shared bank conflicts"),
]


def kernel(path: str, alg_bytes: float) -> str:
    """Markdown of one launch of a `ncu --set full` report exported with
    `ncu -i REPORT --page raw --csv`: the metrics above, the top warp stall reasons, and the
    achieved algorithmic bandwidth (alg_bytes / duration)."""
    lines = open(path).read().splitlines()
    start = next(k for k, line in enumerate(lines) if line.startswith('"ID"'))
    rs = list(csv.reader(io.StringIO("\n".join(lines[start:]))))
    head, units, row = rs[0], rs[1], rs[2]
    col = {h: i for i, h in enumerate(head)}

    def val(m):
        v = row[col[m]].replace(",", "")
        return float(v) if v else 0.0

    out = [f"Kernel: `{kernel_name(row[col['Kernel Name']])}`", "", "| metric | value | unit |", "|---|---|---|"]
    for m, name in KERNEL_METRICS:
        if m in col:
            out.append(f"| {name} (`{m}`) | {row[col[m]]} | {units[col[m]]} |")
    stalls = sorted(((val(h), h) for h in head if h.startswith("smsp__average_warps_issue_stalled_")
                     and h.endswith("_per_issue_active.ratio")), reverse=True)[:6]
    out += ["", "Top warp stalls (cycles per issued instruction): " + ", ".join(
        f"{h.replace('smsp__average_warps_issue_stalled_', '').replace('_per_issue_active.ratio', '')} "
        f"{v:.2f}" for v, h in stalls)]
    dur = val("gpu__time_duration.sum")
    unit = units[col["gpu__time_duration.sum"]]
    dur_s = dur * {"nsecond": 1e-9, "ns": 1e-9, "usecond": 1e-6, "us": 1e-6, "msecond": 1e-3,
                     "ms": 1e-3}.get(unit, 1e-9)
    if alg_bytes > 0 and dur_s > 0:
        out.append(f"Algorithmic bytes {alg_bytes / 1e6:.1f} MB / {dur_s * 1e6:.1f} µs = "
                   f"{alg_bytes / dur_s / 1e9:.0f} GB/s under the profiler (cold L2, clocks as found).")
    return "\n".join(out)


def main(argv: list) -> None:
    if argv[0] == "launches":
        print(launches(argv[1]))
    elif argv[0] == "first-step":  # launch index for ncu -s: the frames after the trials
        print(first_step_after_tuning([k for k, _ in _durations(argv[1])]))
    elif argv[0] == "kernel":
        print(kernel(argv[1], float(argv[2]) if len(argv) > 2 else 0.0))
    elif argv[0] == "traffic":
        kern = traffic(argv[1])
        json.dump({"csrc_hash": csrc_hash(), "source": os.path.basename(argv[1]),
                   "unit": "bytes per launch (dram read + write)", "kernels": kern},
                  open(argv[2], "w"), indent=1)
        print(json.dumps(kern, indent=1))
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
