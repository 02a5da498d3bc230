"""Benchmark of the DS-PHD/MIB filter hot path on B300.

Workload: the automotive-size filter -- 1024x1024 grid at 0.1 m, 4,194,304 persistent +
1,048,576 newborn particles per frame, seeded synthetic lidar scene (30 moving rectangles,
200 static boxes, 2,160 beams), dt = 0.1 s.  A step is one full recursion (Alg. 1-7) on one
frame's measurement grid: dog_set_measurement_grid + dog_step.

Prints one JSON line.  `value` is particle-updates/s (persistent particles x steps / time)
over K timed steps with the grids already resident in HBM (particle state 168 MB > L2, so
no L2 flush is needed); `e2e` is the same metric through the C ABI with host buffers (the
grid copied from pinned host memory and the occupancy and velocity grids read back every
step); `roofline` reports the dominant kernel's achieved bandwidth from per-kernel CUDA
events (a second timed region with DOG_PROFILE); `cpu_baseline` times the CPU oracle on a
bounded sample.  With --impl reference the CPU oracle itself is timed as the reference arm.
Under torchrun each rank runs an independent replica (the filter does not shard).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1605_02406_b300 import scene  # noqa: E402

METRIC = "particle-updates/s at 1024² grid, 4M particles; p50/p99 latency batched vs plain"
CFG_ID = "automotive_1024"

# algorithmic bytes per launch of each kernel: (bytes per persistent particle, per newborn
# slot, per cell): the unique bytes each kernel must move, one read or write per datum
ALG_BYTES = {
    "k_predict": (44, 0, 0),      # read source index 4 + its record 16; write record, w, key
    "k_sort_pass0": (12, 0, 0),   # read cell index 4; write (index, particle) pair 8
    "k_sort_pass1": (16, 0, 0),   # read pair 8; write pair 8
    "k_sort_pass2": (16, 0, 0),
    # read key 4 + perm 4 + gathered record 16 (the weight follows from the out-of-grid flag
    # after a resampled frame); write sorted copy 20
    "k_segsum": (44, 0, 0),
    # lidar: read the cell record 32 (S, tag, 5 moment sums), m_F, z_O, z_F 12; write 6 cell
    # fields 24 (m_O, m_F, rho_b, rho_p, p_occ, mu_UA) and the 5 velocity moments 20
    "k_cell": (0, 0, 88),
    "k_birth": (0, 20, 0),        # write newborn state 16 + weight 4
    "k_normalise": (12, 0, 0),    # lidar, persistent sources: read key 4, w 4, write w' 4
    "k_resample": (8, 4, 0),      # read w' 4; write the source index 4; newborn w 4
}


def csrc_hash() -> str:
    """Hash of the CUDA sources: DRAM traffic recorded in profiles/ncu_traffic.json is
    reported only while the kernels it was measured on are unchanged."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1605_02406_b300", "csrc")
    for n in sorted(os.listdir(d)):
        with open(os.path.join(d, n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _ncu_rows(path: str) -> list:
    """The rows of an ``ncu --csv --log-file`` log (the profiler's own lines skipped)."""
    import csv
    import io
    lines = open(path).read().splitlines()
    start = next(k for k, line in enumerate(lines) if line.startswith('"ID"'))
    return list(csv.DictReader(io.StringIO("\n".join(lines[start:]))))


def _ncu_kernel(full: str) -> str:
    """'void k_segsum<0>(dog::KParams, ...)' -> 'k_segsum'"""
    n = full.split("(")[0].replace("void ", "").replace("<unnamed>::", "").strip()
    return n.split("<")[0].split("::")[-1]


# per-launch labels, in launch order within one frame, of the kernels a frame runs more than
# once or under another name than bench.py's per-kernel times (2-pass sort)
NCU_LABELS = {"k_sort_pass": ["k_sort_pass0", "k_sort_pass1"],
              "k_sort_offsets": ["k_sort_offsets0", "k_sort_offsets1"],
              "k_sort_count": ["k_sort_count1"], "k_scan_tiles": ["k_scan_births", "k_scan_cdf"],
              "k_segsum_lidar": ["k_segsum"], "k_normalise_lidar": ["k_normalise"]}


def write_ncu_traffic(paths: list, out: str) -> dict:
    """DRAM bytes per launch (``--metrics dram__bytes_read.sum,dram__bytes_write.sum``, one
    frame's launches of each kernel) into ``out``, tagged with the hash of the CUDA sources."""
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    launches = {}
    for j, p in enumerate(paths):
        for r in _ncu_rows(p):
            if r["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                d = launches.setdefault((j, int(r["ID"])), {"kernel": _ncu_kernel(r["Kernel Name"])})
                d[r["Metric Name"].split(".")[0].rsplit("_", 1)[1]] = \
                    float(r["Metric Value"].replace(",", "")) * scale.get(r["Metric Unit"], 1)
    by_kernel = {}
    for i in sorted(launches):
        by_kernel.setdefault(launches[i]["kernel"], []).append(launches[i])
    rw = {}
    for k, ls in by_kernel.items():
        labels = NCU_LABELS.get(k, [k])
        if len(ls) != len(labels):
            raise SystemExit(f"{k}: {len(ls)} launches captured, one frame has {len(labels)}")
        for lab, d in zip(labels, ls):
            rw[lab] = {"read": d["read"], "write": d["write"]}
    js = {"csrc_hash": csrc_hash(), "unit": "bytes per launch (dram read + write)",
          "kernels": {k: v["read"] + v["write"] for k, v in rw.items()}, "read_write": rw}
    with open(out, "w") as fh:
        json.dump(js, fh, indent=1)
    return js


def ncu_launch_table(path: str) -> str:
    """Per kernel: launches, total and mean device time and share, from a
    ``--metrics gpu__time_duration.sum --csv`` log (markdown)."""
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    tot = {}
    for r in _ncu_rows(path):
        if r["Metric Name"] == "gpu__time_duration.sum":
            k = _ncu_kernel(r["Kernel Name"])
            us = float(r["Metric Value"].replace(",", "")) * scale.get(r["Metric Unit"], 1.0)
            n, t = tot.get(k, (0, 0.0))
            tot[k] = (n + 1, t + us)
    allt = sum(t for _, t in tot.values())
    lines = ["| kernel | launches | total µs | µs / launch | share |", "|---|---|---|---|---|"]
    for k, (n, t) in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        lines.append(f"| {k} | {n} | {t:.1f} | {t / n:.1f} | {100 * t / allt:.1f} % |")
    lines.append(f"| **all** | {sum(n for n, _ in tot.values())} | {allt:.1f} | | 100 % |")
    return "\n".join(lines)


def peaks() -> tuple:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.f = tempfile.NamedTemporaryFile("w+", delete=False)
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # the sampler is running before the timed region starts
        except OSError:
            self.p = None

    def start(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if self.t0 is not None and not (self.t0 - 0.05 <= ts <= self.t1 + 0.05):
                    continue
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 4 + k and r[4 + k].strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu() -> dict:
    """The host's core count and CPU model (the oracle runs on one of its cores)."""
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_frames(params: dict, grids: list, mode: str, frames: int, budget_s: float = 1e9) -> tuple:
    """Frames of the oracle from the initial state (grid set + step, wall clock); returns
    (frames done, seconds)."""
    from oracle import OracleFilter
    o = OracleFilter(params, mode)
    n, el = 0, 0.0
    while n < frames and el < budget_s:
        g = grids[n % len(grids)]
        args = [g["m_occ"], g["m_free"]] + ([g["p_A"], g["z_vr"], g["sigma_vr"]] if "p_A" in g else [])
        o.set_measurement_grid(*args)
        t0 = time.perf_counter()
        o.step(0.1)
        el += time.perf_counter() - t0
        n += 1
    return n, el


def cpu_oracle_rate(params: dict, grids: list, budget_s: float = 12.0) -> dict:
    """The oracle (FP32 mirror) on frames of the same workload until about budget_s, and
    its binary64 mode on a few frames."""
    n, el = oracle_frames(params, grids, "f32", len(grids), budget_s)
    n64, el64 = oracle_frames(params, grids, "f64", 3, budget_s / 2)
    return {"value": params["nu"] * n / el, "unit": "particle-updates/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{n} consecutive frames of the full 1024x1024 / 4,194,304 + 1,048,576 "
                      f"particle workload from the initial state, single thread (step time only)",
            "f64": {"value": params["nu"] * n64 / el64, "frames": n64},
            "host": host_cpu()}


def cpu_plan() -> dict:
    """The CPU baseline plan: both oracle modes, single thread, median of 3 runs, on the plain
    128x128 workload (20 frames), the automotive 1024x1024 workload (100 frames), the first 10
    frames of the 2048x2048 lidar + radar workload and 3 sampled filters of the 64-filter batch
    (50 frames each).  Step time only (scene generation excluded).  Tens of minutes."""
    cases = [("plain_128", scene.CONFIGS["plain_128"], 20, 1001),
             ("automotive_1024", scene.CONFIGS["automotive_1024"], 100, 1002),
             ("fusion_2048 (first 10 frames)", scene.CONFIGS["fusion_2048"], 10, 1005)]
    bcfgs = scene.batched_configs(64)
    for k in (0, 21, 42):
        cases.append((f"batched filter {k} ({bcfgs[k]['width']}x{bcfgs[k]['height']}, {bcfgs[k]['nu']:,} particles)",
                      bcfgs[k], 50, 2000 + k))
    out = {"host": host_cpu(), "runs": 3, "cases": []}
    for name, cfg, frames, seed in cases:
        params = scene.filter_params(cfg, seed=42)
        grids = scene.frame_sequence(cfg, min(frames, 16), seed)
        row = {"workload": name, "frames": frames, "num_particles": params["nu"]}
        for mode in ("f32", "f64"):
            ts = [oracle_frames(params, grids, mode, frames)[1] for _ in range(3)]
            t = statistics.median(ts)
            row[mode] = {"seconds": t, "particle_updates_per_s": params["nu"] * frames / t}
        out["cases"].append(row)
        print(json.dumps(row), flush=True)
    return out


def bench_config(cfg: dict, params: dict, world: int) -> dict:
    """The workload description, the same in both arms."""
    return {"workload": cfg["name"], "grid": "1024x1024", "cell_size_m": 0.1,
            "num_particles": params["nu"], "num_birth": params["nu_b"],
            "scene": "30 moving rectangles, 200 static boxes, 2160 beams",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (particle state 168 MB); no flush"}


def run_reference(args) -> None:
    """Reference arm: the CPU oracle, one full frame of the workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import OracleFilter
    cfg = scene.CONFIGS[CFG_ID]
    params = scene.filter_params(cfg)
    grids = scene.frame_sequence(cfg, min(args.steps + args.warmup, 16), 1002)
    o = OracleFilter(params, "f32")
    warm = args.warmup
    for k in range(warm):
        g = grids[k % len(grids)]
        o.set_measurement_grid(g["m_occ"], g["m_free"])
        o.step(0.1)
    # bounded sample: full frames of the workload, at most args.steps and about 120 s
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        g = grids[(warm + done) % len(grids)]
        o.set_measurement_grid(g["m_occ"], g["m_free"])
        o.step(0.1)
        done += 1
        if time.perf_counter() - t0 > 120.0:
            break
    el = time.perf_counter() - t0
    v = params["nu"] * done / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "particle-updates/s",
        "n_gpus": args.gpus, "steps": done, "warmup": warm,
        "ms_per_step": el / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(cfg, params, 1),
        "cpu_baseline": {"value": v, "unit": "particle-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{done} full frames (of {args.steps} requested, bounded to "
                                   f"~120 s) after {warm} warm-up frames, single thread"},
        "e2e": {"value": v, "unit": "particle-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def batched_latency(frames: int, warmup: int, dt: float = 0.1, rank: int = 0, world: int = 1) -> dict:
    """p50/p99 GPU time of one frame of the 64-filter batched workload (uneven grids and
    particle counts), stepped by a plain loop of dog_step calls vs one dog_batch_step.
    Under several ranks each rank steps the filters placed on it by their HBM need; the
    times are the slowest rank's, the throughput all filters' particles per that time."""
    import torch

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300 import replicas
    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    cfgs_all = scene.batched_configs(64)
    need = [N.dog_workspace_bytes(N.make_params(scene.filter_params(c))) for c in cfgs_all]
    where = replicas.place_by_budget(need, world, 100e9)
    mine = [(k, c) for k, (c, r) in enumerate(zip(cfgs_all, where)) if r == rank]
    shared = torch.cuda.Stream()
    filters = []
    for k, c in mine:
        f = DogFilter(scene.filter_params(c, seed=100 + k), stream=shared)
        g = scene.frame_sequence(c, 1, 2000 + k)[0]
        f.set_measurement_grid(**{kk: torch.tensor(v, device="cuda") for kk, v in g.items()})
        filters.append(f)
    # each filter's sort configuration picked by dog_autotune on its first frame, before the
    # batch captures them
    for f in filters:
        f.step(dt)
        f.autotune()
    dts = [dt] * len(filters)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * frames)]

    def run(step):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        for k in range(frames):
            ev[2 * k].record(shared)
            step()
            ev[2 * k + 1].record(shared)
        torch.cuda.synchronize()
        return [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(frames)]

    def plain():
        for f in filters:
            f.step(dt)

    t_plain = t_batch = [0.0]  # a rank without filters still joins the reductions
    grouping = None
    if filters:
        batch = DogBatch(filters)
        grouping = batch.autotune(dts, frames=2)  # real frames, before the timed region
        t_plain = run(plain)
        t_batch = run(lambda: batch.step(dts))
        batch.close()
    nu_total = sum(int(c["nu"]) for c in cfgs_all)
    for f in filters:
        f.close()
    pct = {k: replicas.slowest(float(np.percentile(t, q)), "cuda")
           for k, t, q in (("plain_p50", t_plain, 50), ("plain_p99", t_plain, 99),
                           ("batched_p50", t_batch, 50), ("batched_p99", t_batch, 99))}
    med = replicas.slowest(float(np.median(t_batch)), "cuda")
    return dict({"workload": "batched: 64 filters, sides 256-1024 at 0.1 m, 2^18-2^22 particles each "
                             f"({nu_total:,} in total)" + (f", placed on {world} GPUs by HBM need" if world > 1 else ""),
                 "frames": frames, "grouping": grouping}, **pct,
                batched_particle_updates_per_s=nu_total / (med * 1e-3))


def small_batch_latency(frames: int, warmup: int, n: int = 128, side: int = 64, nu: int = 8192) -> dict:
    """Many small filters (128 grids of 64x64 at 0.25 m, 8,192 + 2,048 particles each), where
    launches rather than bytes dominate: a loop of dog_step calls vs one batched frame."""
    import torch

    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    shared = torch.cuda.Stream()
    rng = np.random.default_rng(3)
    filters = []
    for k in range(n):
        p = dict(width=side, height=side, cell_size=0.25, nu=nu, nu_b=nu // 4, p_S=0.99, p_B=0.02,
                 alpha=0.9, sigma_pos=0.05, sigma_vel=1.0, sigma_birth_vel=4.0, sensor_x=side * 0.125,
                 sensor_y=side * 0.125, seed=700 + k, flags=0)
        f = DogFilter(p, stream=shared)
        g = scene.random_measurement_grid(side, side, rng)
        f.set_measurement_grid(**{kk: torch.tensor(v, device="cuda") for kk, v in g.items()})
        filters.append(f)
    batch = DogBatch(filters)
    grouping = batch.autotune(0.1, frames=2)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * frames)]

    def run(step):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        for k in range(frames):
            ev[2 * k].record(shared)
            step()
            ev[2 * k + 1].record(shared)
        torch.cuda.synchronize()
        return [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(frames)]

    t_plain = run(lambda: [f.step(0.1) for f in filters])
    t_batch = run(lambda: batch.step(0.1))
    batch.close()
    for f in filters:
        f.close()
    return {"workload": f"{n} filters of {side}x{side} at 0.25 m, {nu:,} + {nu // 4:,} particles each",
            "grouping": grouping,
            "plain_p50": float(np.percentile(t_plain, 50)), "plain_p99": float(np.percentile(t_plain, 99)),
            "batched_p50": float(np.percentile(t_batch, 50)), "batched_p99": float(np.percentile(t_batch, 99))}


def evaluation_time(reps: int = 50) -> dict:
    """Device time of the evaluation calls (cluster statistics of every object and the
    Mahalanobis static/dynamic classification over 42 thresholds) on the 1024x1024 grid."""
    import torch

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.evaluate import Evaluator
    from paper_1605_02406_b300.filter import DogFilter
    cfg = scene.CONFIGS[CFG_ID]
    seq = scene.frame_sequence_with_truth(cfg, 4, 1002)
    f = DogFilter(scene.filter_params(cfg))
    for g, _ in seq:
        f.set_measurement_grid(**g)
        f.step(cfg["dt"])
    truth = seq[-1][1]
    thr = np.concatenate([[0.0], np.logspace(-2, 3, 41)])
    ev = Evaluator(f, len(truth["velocity"]), thr)
    obj = torch.as_tensor(truth["object"], device="cuda")
    lab = torch.as_tensor(truth["dynamic"], device="cuda")
    f.stream.wait_stream(torch.cuda.current_stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def once():
        N.dog_eval_clusters(f.h, obj.data_ptr(), ev.n_objects, ev.scratch.data_ptr(), ev.stats.data_ptr())
        N.dog_eval_mahalanobis(f.h, lab.data_ptr(), 0.5, ev.thr.data_ptr(), len(ev.thr),
                               ev.counts.data_ptr(), 0)
    for _ in range(3):
        once()
    f.sync()
    e0.record(f.stream)
    for _ in range(reps):
        once()
    e1.record(f.stream)
    f.sync()
    us = e0.elapsed_time(e1) / reps * 1e3
    out = {"grid": "1024x1024", "objects": int(ev.n_objects), "thresholds": len(thr),
           "us_per_evaluation": us, "cells_per_s": f.C / (us * 1e-6)}
    f.close()
    return out


def fusion_rate(steps: int, warmup: int) -> dict:
    """Device-resident step rate of the lidar + radar workload (2048x2048 at 0.1 m,
    16,777,216 + 4,194,304 particles, 64 radar detections a frame)."""
    import torch

    from paper_1605_02406_b300.filter import DogFilter
    cfg = scene.CONFIGS["fusion_2048"]
    params = scene.filter_params(cfg, seed=42)
    grids = scene.frame_sequence(cfg, 8, 1005)
    dev = [{k: torch.tensor(v, device="cuda") for k, v in g.items()} for g in grids]
    f = DogFilter(params)
    for k in range(warmup):
        f.set_measurement_grid(**dev[k % 8])
        f.step(cfg["dt"])
    f.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(f.stream)
    for k in range(steps):
        f.set_measurement_grid(**dev[(warmup + k) % 8])
        f.step(cfg["dt"])
    e1.record(f.stream)
    f.sync()
    ms = e0.elapsed_time(e1) / steps
    f.close()
    return {"workload": cfg["name"], "steps": steps, "ms_per_step": ms,
            "value": params["nu"] / (ms * 1e-3), "unit": "particle-updates/s"}


def ego_rate(steps: int, warmup: int) -> dict:
    """Device-resident step rate of the 1024x1024 workload with ego-motion compensation
    every frame (vehicle at 10 m/s turning at 0.2 rad/s: 1 m and 0.02 rad a frame), next
    to the same filter without it."""
    import torch

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogFilter
    cfg = scene.CONFIGS["automotive_1024"]
    grids = scene.frame_sequence(cfg, 8, 1002)
    dev = [{k: torch.tensor(v, device="cuda") for k, v in g.items()} for g in grids]
    out = {"workload": cfg["name"] + ", ego motion 1 m and 0.02 rad a frame", "steps": steps}
    for name, flags in (("ego", N.DOG_EGO), ("plain", 0)):
        f = DogFilter(scene.filter_params(cfg, flags=flags))

        def frame(k):
            f.set_measurement_grid(**dev[k % 8])
            if flags:
                f.set_ego_motion(1.0, 0.0, 0.02)
            f.step(cfg["dt"])

        for k in range(warmup):
            frame(k)
        f.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(f.stream)
        for k in range(steps):
            frame(warmup + k)
        e1.record(f.stream)
        f.sync()
        out[name + "_ms_per_step"] = e0.elapsed_time(e1) / steps
        f.close()
    out["value"] = cfg["nu"] / (out["ego_ms_per_step"] * 1e-3)
    out["unit"] = "particle-updates/s"
    return out


def phdmib_rate(steps: int, warmup: int) -> dict:
    """Device-resident step rate of the PHD/MIB filter (Sect. VI) on the 1024x1024 workload,
    its Bernoulli grids derived from the same lidar scenes (scene.bernoulli_grid)."""
    import torch

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogFilter
    cfg = scene.CONFIGS["automotive_1024"]
    grids = [scene.bernoulli_grid(g) for g in scene.frame_sequence(cfg, 8, 1002)]
    dev = [{k: torch.tensor(v, device="cuda") for k, v in g.items()} for g in grids]
    params = scene.filter_params(cfg, flags=N.DOG_FULL)
    f = DogFilter(params)
    for k in range(warmup):
        f.set_bernoulli_grid(**dev[k % 8])
        f.step(cfg["dt"])
    f.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(f.stream)
    for k in range(steps):
        f.set_bernoulli_grid(**dev[(warmup + k) % 8])
        f.step(cfg["dt"])
    e1.record(f.stream)
    f.sync()
    ms = e0.elapsed_time(e1) / steps
    f.close()
    return {"workload": cfg["name"] + ", PHD/MIB filter (Bernoulli observation)", "steps": steps,
            "ms_per_step": ms, "value": params["nu"] / (ms * 1e-3), "unit": "particle-updates/s"}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-filter latency run")
    ap.add_argument("--no-fusion", action="store_true", help="skip the lidar + radar workload")
    ap.add_argument("--no-evaluation", action="store_true", help="skip timing the evaluation calls")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop runs")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="simulated seconds of arrivals per serving arm (the workload states 60)")
    ap.add_argument("--no-ego", action="store_true", help="skip the ego-motion workload")
    ap.add_argument("--no-phdmib", action="store_true", help="skip the PHD/MIB filter workload")
    ap.add_argument("--cpu-plan", action="store_true", help="only the full CPU baseline plan (slow)")
    ap.add_argument("--ncu-traffic", nargs="+", metavar="CSV",
                    help="write profiles/ncu_traffic.json from ncu DRAM-byte logs and exit")
    ap.add_argument("--ncu-launches", metavar="CSV", help="print the per-kernel launch table of an ncu log and exit")
    args = ap.parse_args()
    if args.ncu_traffic:
        js = write_ncu_traffic(args.ncu_traffic, os.path.join(ROOT, "profiles", "ncu_traffic.json"))
        for k, v in js["read_write"].items():
            print(f"{k:18s} read {v['read'] / 1e6:8.1f} MB  write {v['write'] / 1e6:8.1f} MB")
        return
    if args.ncu_launches:
        print(ncu_launch_table(args.ncu_launches))
        return
    if args.cpu_plan:
        print(json.dumps(cpu_plan()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    import torch.distributed as dist

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogFilter

    from paper_1605_02406_b300 import replicas
    world, rank, local = replicas.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    cfg = scene.CONFIGS[CFG_ID]
    params = scene.filter_params(cfg, seed=replicas.replica_seed(42, rank))
    n_grids = min(args.steps + args.warmup, 24)
    grids = scene.frame_sequence(cfg, n_grids, 1002)
    dev_grids = [{k: torch.tensor(v, device="cuda") for k, v in g.items()} for g in grids]

    # ---------------------------------------------------------------- device-resident run
    # the sort's configuration is picked by dog_autotune on the first frame's keys (before
    # the timed region); filters created later in this size class start from that choice
    params = dict(params, flags=params.get("flags", 0) | N.DOG_AUTOTUNE)
    f = DogFilter(params)
    st = f.stream
    for k in range(args.warmup):
        f.set_measurement_grid(**dev_grids[k % n_grids])
        f.step(cfg["dt"])
        if k == 0:
            sort_cfg = f.autotune()
    f.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    # the timed loop calls the C ABI directly (grid pointers prepared here, the grids already
    # on the device and ordered before the filter's stream), so that the host stays ahead of
    # the GPU from the first step on
    f.stream.wait_stream(torch.cuda.current_stream())
    grid_ptrs = [{k: v.data_ptr() for k, v in g.items()} for g in dev_grids]
    gc.collect()
    gc.disable()
    clk = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    ev[0].record(st)
    for k in range(args.steps):
        N.dog_set_measurement_grid(f.h, grid_ptrs[(args.warmup + k) % n_grids], N.DOG_DEVICE)
        N.dog_step(f.h, cfg["dt"])
        ev[k + 1].record(st)
    f.sync()
    torch.cuda.synchronize()
    clk.end()
    gc.enable()
    barrier()
    clocks = clk.stop()
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms_total = ev[0].elapsed_time(ev[-1])
    ms_max = replicas.slowest(ms_total, "cuda")
    value = world * params["nu"] * args.steps / (ms_max * 1e-3)
    launches = args.steps * (f.kernels_per_step() + 1)  # + the grid take-over kernel
    cells_check = f.cells(["m_occ"])["m_occ"]
    assert np.isfinite(cells_check).all()
    f.close()

    # ------------------------------------------------------------- end-to-end, host buffers
    fe = DogFilter(params)
    C = params["width"] * params["height"]
    pin = [{k: torch.from_numpy(v).pin_memory() for k, v in g.items()} for g in grids]
    out = {k: torch.empty(C, dtype=torch.float32).pin_memory() for k in ("p_occ", "mean_vx", "mean_vy")}

    out2 = [out, {k: torch.empty(C, dtype=torch.float32).pin_memory() for k in out}]

    def upload(k):
        g = pin[k % n_grids]  # each frame has its own pinned buffers, reused frames later
        N.dog_set_measurement_grid(fe.h, {kk: v.data_ptr() for kk, v in g.items()}, N.DOG_HOST_ASYNC)

    def e2e_step(k):
        # step frame k (its grid is already uploaded or on its way), upload frame k + 1 so
        # that the copy overlaps frame k on the GPU, then start reading frame k's cells back;
        # the read-back of frame k - 1 is complete when that call returns
        N.dog_step(fe.h, cfg["dt"])
        upload(k + 1)
        N.dog_get_cells_async(fe.h, {kk: v.data_ptr() for kk, v in out2[k % 2].items()})

    upload(0)
    for k in range(args.warmup):
        e2e_step(k)
    N.dog_wait_cells(fe.h)
    torch.cuda.synchronize()
    barrier()
    # 100 steps whatever --steps is (about 35 ms): the last frame's read-back, which nothing
    # overlaps, and the host's jitter then weigh what they weigh in a stream of frames
    ke = 100
    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    for k in range(ke):
        e2e_step(args.warmup + k)
    N.dog_wait_cells(fe.h)  # the last frame's cells are on the host
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    gc.enable()
    e2e_value = replicas.job_throughput(params["nu"] * ke, e2e_s, "cuda")
    fe.close()

    # ------------------------------------------------------ per-kernel events (roofline)
    fp = DogFilter(dict(params, flags=N.DOG_PROFILE))
    for k in range(args.warmup):
        fp.set_measurement_grid(**dev_grids[k % n_grids])
        fp.step(cfg["dt"])
    fp.sync()
    fp.profile()
    kp = min(args.steps, 30)
    for k in range(kp):
        fp.set_measurement_grid(**dev_grids[(args.warmup + k) % n_grids])
        fp.step(cfg["dt"])
    prof, nsteps = fp.profile()
    fp.close()
    per_kernel_us = {k: v / max(nsteps, 1) * 1e3 for k, v in prof.items()}
    nu, nb = params["nu"], params["nu_b"]
    kern_gbs = {}
    for k, us in per_kernel_us.items():
        a, b, c = ALG_BYTES.get(k, (0, 0, 0))
        byts = a * nu + b * nb + c * C
        kern_gbs[k] = byts / (us * 1e-6) / 1e9 if us > 0 and byts else None
    # dominant kernel: the longest one that moves algorithmic bytes (the scans move ~none)
    dom = max((k for k in per_kernel_us if kern_gbs.get(k)), key=lambda k: per_kernel_us[k])
    peak, peak_kind = peaks()
    a, b, c = ALG_BYTES[dom]
    alg = a * nu + b * nb + c * C
    traffic = None
    tf = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tf):
        tj = json.load(open(tf))
        if tj.get("csrc_hash") == csrc_hash() and dom in tj.get("kernels", {}):
            traffic = tj["kernels"][dom]
    achieved = kern_gbs[dom]

    # workloads of independent filters: split over the ranks by HBM need, combined here
    batched = {"workload": None}
    if not args.no_batched:
        batched = batched_latency(frames=min(args.steps, 50), warmup=args.warmup, rank=rank, world=world)
    serving = serving_plain = None
    if not args.no_serving:
        from paper_1605_02406_b300 import serve
        serving_plain = serve.run(seconds=args.serving_seconds, rank=rank, world=world, plain=True)
        serving = serve.run(seconds=args.serving_seconds, rank=rank, world=world)
        if world > 1:
            last = replicas.slowest(serving["last_completion_s"], "cuda")
            updates = replicas.total(serving["updates"], "cuda")
            serving.update(
                streams_admitted=int(replicas.total(serving["streams_admitted"], "cuda")),
                workspace_gb=replicas.total(serving["workspace_gb"], "cuda"),
                requests=int(replicas.total(serving["requests"], "cuda")),
                offered_particle_updates_per_s=replicas.total(serving["offered_particle_updates_per_s"], "cuda"),
                served_particle_updates_per_s=updates / last,
                latency_ms={k: replicas.slowest(v, "cuda") for k, v in serving["latency_ms"].items()},
                workload=serving["workload"] + f" per GPU, {world} GPUs (slowest rank's latencies)")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    # streams that come and go, admitted as others leave (rank 0 alone: a per-GPU figure)
    sessions = None
    if not args.no_serving:
        from paper_1605_02406_b300 import serve
        sessions = serve.run_sessions(seconds=min(args.serving_seconds, 5.0))
        if world > 1:
            sessions["workload"] += " (rank 0's GPU only)"
    small = None
    if not args.no_batched:
        small = small_batch_latency(frames=min(args.steps, 50), warmup=args.warmup)
    evaluation = None if args.no_evaluation else evaluation_time()
    fusion = None
    if not args.no_fusion:
        fusion = fusion_rate(steps=min(args.steps, 100), warmup=args.warmup)
    ego = None if args.no_ego else ego_rate(steps=min(args.steps, 200), warmup=args.warmup)
    phdmib = None if args.no_phdmib else phdmib_rate(steps=min(args.steps, 200), warmup=args.warmup)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(scene.filter_params(cfg), grids[:8])
    line = {
        "metric": METRIC, "value": value, "unit": "particle-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(cfg, params, world),
        "launch": "CUDA graph per step",
        "sort": dict(sort_cfg, chosen_by="dog_autotune"),
        "e2e": {"value": e2e_value, "unit": "particle-updates/s", "steps": ke,
                "h2d_bytes_per_step": 2 * 4 * C, "d2h_bytes_per_step": 3 * 4 * C},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": traffic, "algorithmic_bytes": alg,
                     "timing": "per-kernel CUDA events, DOG_PROFILE region of "
                               f"{nsteps} steps (kernels launched one by one)"},
        "kernels_us": {k: round(v, 2) for k, v in per_kernel_us.items()},
        "kernels_gbs": {k: (round(v, 1) if v else None) for k, v in kern_gbs.items()},
        "clocks": clocks,
        "cpu_baseline": cpu,
        "fusion": fusion,
        "ego": ego,
        "phdmib": phdmib,
        "evaluation": evaluation,
        "serving_sessions": sessions,
        "serving_plain": serving_plain,
        "serving": serving,
        # last, so that the tail of the line the driver keeps holds it: per-frame latency of
        # the 64-filter batched workload (a loop of dog_step vs one batched frame), of the
        # many-small-filters batch, and of the single filter's step
        "latency_ms": dict(batched, step_p50=float(np.percentile(per_step, 50)),
                           step_p99=float(np.percentile(per_step, 99)), small_filters=small),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
