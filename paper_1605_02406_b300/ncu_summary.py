"""Summaries of Nsight Compute CSV logs of the filter's kernels.

    python -m paper_1605_02406_b300.ncu_summary launches LOG.csv      # markdown table
    python -m paper_1605_02406_b300.ncu_summary traffic LOG.csv OUT.json --steps-from LOG

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
    """'void k_segsum<0>(dog::KParams, ...)' -> 'k_segsum'"""
    n = full.split("(")[0].replace("void ", "").strip()
    return n.split("<")[0].split("::")[-1]


def launches(path: str) -> str:
    n = collections.Counter()
    t = collections.defaultdict(float)
    for r in rows(path):
        if r["Metric Name"] != "gpu__time_duration.sum":
            continue
        k = kernel_name(r["Kernel Name"])
        scale = {"ns": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}.get(r["Metric Unit"], 1e-3)
        n[k] += 1
        t[k] += float(r["Metric Value"].replace(",", "")) * scale
    total = sum(t.values())
    out = ["| kernel | launches | total µs | µs / launch | share |", "|---|---|---|---|---|"]
    for k in sorted(t, key=lambda k: -t[k]):
        out.append(f"| {k} | {n[k]} | {t[k]:.1f} | {t[k] / n[k]:.1f} | {100 * t[k] / total:.1f} % |")
    out.append(f"| **all** | {sum(n.values())} | {total:.1f} | | 100 % |")
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


def main(argv: list) -> None:
    if argv[0] == "launches":
        print(launches(argv[1]))
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
