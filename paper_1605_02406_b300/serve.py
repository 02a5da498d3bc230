"""Serving loop: many independent filter streams on one GPU, requests arriving over time.

Each stream is a filter (grid side 256/512/1024 at 0.1 m, 16 particles per cell, newborn
= a quarter); a request is one frame of one stream (its measurement grid is already on the
device) and must see the stream's earlier frames, so a stream's requests run in order.
Streams are admitted in order while their workspaces fit the HBM budget.  Requests arrive
by independent Poisson processes (10 Hz per stream); the loop issues every request whose
arrival time has passed on its stream's own CUDA stream, so requests of different streams
overlap on the GPU, and stamps its completion with a CUDA event.  Latency = completion -
arrival on the GPU's clock (the arrivals are mapped onto it through an event recorded at
the start).

    python -m paper_1605_02406_b300.serve --seconds 3
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import native as N
from . import replicas, scene
from .filter import DogFilter


def admit(cfgs: list, budget_bytes: float, rank: int = 0, world: int = 1) -> tuple:
    """Streams placed on this rank by their workspaces against a budget per rank (one rank:
    admitted in order while they fit); also the number rejected on every rank and the bytes
    used on this one."""
    need = [N.dog_workspace_bytes(N.make_params(scene.filter_params(c))) + 8 * c["width"] * c["height"]
            for c in cfgs]  # + the grid
    where = replicas.place_by_budget(need, world, budget_bytes)
    admitted = [dict(c, index=k) for k, (c, r) in enumerate(zip(cfgs, where)) if r == rank]
    used = sum(b for b, r in zip(need, where) if r == rank)
    return admitted, sum(1 for r in where if r < 0), used


def run(n_streams: int = 256, seconds: float = 3.0, budget_gb: float = 120.0, seed: int = 7,
        warm_frames: int = 2, rank: int = 0, world: int = 1) -> dict:
    """One rank's share of the serving workload (all of it on one rank); budget_gb is per
    rank.  Besides the rates and latency percentiles, returns the raw counts (updates, the
    last completion) from which several ranks' results combine."""
    cfgs = scene.serving_stream_configs(n_streams)
    admitted, rejected, used = admit(cfgs, budget_gb * 1e9, rank, world)
    rng = np.random.default_rng(seed + rank)
    filters, grids = [], []
    for c in admitted:
        f = DogFilter(scene.filter_params(c, seed=500 + c["index"]))
        g = scene.random_measurement_grid(c["width"], c["height"], rng)
        dg = {kk: torch.tensor(v, device="cuda") for kk, v in g.items()}
        f.set_measurement_grid(**dg)
        filters.append(f)
        grids.append(dg)
    for _ in range(warm_frames):  # capture every filter's graph, fill the caches
        for f in filters:
            f.step(0.1)
    torch.cuda.synchronize()
    # arrival times: Poisson at rate_hz per stream over the run
    arrivals = []
    for k, c in enumerate(admitted):
        t = rng.exponential(1.0 / c["rate_hz"])
        while t < seconds:
            arrivals.append((t, k))
            t += rng.exponential(1.0 / c["rate_hz"])
    arrivals.sort()
    start = torch.cuda.Event(enable_timing=True)
    start.record()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = []  # (arrival, stream, event)
    i = 0
    while i < len(arrivals):
        now = time.perf_counter() - t0
        if arrivals[i][0] > now:
            time.sleep(min(arrivals[i][0] - now, 0.0005))
            continue
        while i < len(arrivals) and arrivals[i][0] <= now:
            a, k = arrivals[i]
            f = filters[k]
            f.step(0.1)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(f.stream)
            done.append((a, k, ev))
            i += 1
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = np.array([start.elapsed_time(ev) * 1e-3 - a for a, _, ev in done])
    updates = sum(int(admitted[k]["nu"]) for _, k, _ in done)
    last = max(start.elapsed_time(ev) for _, _, ev in done) * 1e-3
    for f in filters:
        f.close()
    return {
        "workload": f"serving: {n_streams} streams (sides 256/512/1024, 16 particles per cell), "
                    f"Poisson 10 Hz each, {budget_gb:.0f} GB admission",
        "streams_admitted": len(admitted), "streams_rejected": rejected,
        "workspace_gb": used / 1e9, "seconds": seconds, "requests": len(done),
        "offered_particle_updates_per_s": sum(float(c["nu"]) * c["rate_hz"] for c in admitted),
        "served_particle_updates_per_s": updates / last,
        "updates": updates, "last_completion_s": last,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
        "wall_s": wall,
    }


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=256)
    ap.add_argument("--seconds", type=float, default=3.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    print(json.dumps(run(args.streams, args.seconds, args.budget_gb)))


if __name__ == "__main__":
    main()
