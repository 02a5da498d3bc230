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

`run_sessions` is the same loop with streams that come and go: each connects at some time,
waits in arrival order until a slot and its HBM need are free (`Admission`), is served for
a session of random length, and on leaving returns its workspace, so streams that could
not fit at first are admitted as others depart.

    python -m paper_1605_02406_b300.serve --seconds 3
    python -m paper_1605_02406_b300.serve --sessions --seconds 3 --budget-gb 40
"""
from __future__ import annotations

import argparse
import collections
import gc
import json
import queue
import threading
import time

import numpy as np
import torch

from cuda.bindings import runtime as cudart

from . import native as N
from . import replicas, scene
from .filter import DogFilter


def _check(err) -> None:
    if err != cudart.cudaError_t.cudaSuccess:
        raise RuntimeError(f"CUDA runtime: {err}")


class Admission:
    """Admission of streams by HBM need and free slots, in arrival order: a stream waits
    until every stream that arrived before it is admitted and its own need fits the budget
    left by the streams still active (no overtaking, so no stream waits forever behind a
    flow of smaller ones).  Pure host bookkeeping in bytes."""

    def __init__(self, budget_bytes: float, slots: int):
        self.budget, self.slots = float(budget_bytes), int(slots)
        self.used = 0.0
        self.active = {}  # stream -> bytes
        self.queue = collections.deque()

    def request(self, k: int, need: float) -> None:
        if need > self.budget:
            raise ValueError(f"stream {k} needs {need:.0f} bytes, more than the whole budget")
        self.queue.append((k, float(need)))

    def admit(self) -> list:
        """Streams admitted now, in arrival order."""
        out = []
        while (self.queue and len(self.active) < self.slots
               and self.used + self.queue[0][1] <= self.budget):
            k, need = self.queue.popleft()
            self.active[k] = need
            self.used += need
            out.append(k)
        return out

    def release(self, k: int) -> None:
        self.used -= self.active.pop(k)
        if not self.active:
            self.used = 0.0  # no rounding residue once nothing is active


def stream_need(c: dict) -> int:
    """Device bytes of one stream: its filter workspace and its measurement grid."""
    return N.dog_workspace_bytes(N.make_params(scene.filter_params(c))) + 8 * c["width"] * c["height"]


def admit(cfgs: list, budget_bytes: float, rank: int = 0, world: int = 1) -> tuple:
    """Streams placed on this rank by their workspaces against a budget per rank (one rank:
    admitted in order while they fit); also the number rejected on every rank and the bytes
    used on this one."""
    need = [stream_need(c) for c in cfgs]
    where = replicas.place_by_budget(need, world, budget_bytes)
    admitted = [dict(c, index=k) for k, (c, r) in enumerate(zip(cfgs, where)) if r == rank]
    used = sum(b for b, r in zip(need, where) if r == rank)
    return admitted, sum(1 for r in where if r < 0), used


def run(n_streams: int = 256, seconds: float = 3.0, budget_gb: float = 120.0, seed: int = 7,
        warm_frames: int = 2, rank: int = 0, world: int = 1, plain: bool = False) -> dict:
    """One rank's share of the serving workload (all of it on one rank); budget_gb is per
    rank.  Besides the rates and latency percentiles, returns the raw counts (updates, the
    last completion) from which several ranks' results combine.  plain=True is the plain
    per-grid loop on the same streams and arrivals: every filter on one CUDA stream, so the
    requests run one at a time in arrival order (the queue's wait counts in the latency)."""
    cfgs = scene.serving_stream_configs(n_streams)
    admitted, rejected, used = admit(cfgs, budget_gb * 1e9, rank, world)
    rng = np.random.default_rng(seed + rank)
    filters, grids = [], []
    one = torch.cuda.Stream() if plain else None
    for c in admitted:
        f = DogFilter(scene.filter_params(c, seed=500 + c["index"]), stream=one)
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
    # the collector is paused while requests are issued: a collection pass over the loop's
    # objects can hold the host thread for tens of milliseconds, and every request arriving
    # meanwhile would count that wait in its latency.  (Before the start event: the GPU and
    # host clocks of the latencies start together.)
    gc.collect()
    gc.disable()
    try:
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = []  # (arrival, stream, event)
        lag = []
        i = 0
        while i < len(arrivals):
            now = time.perf_counter() - t0
            if arrivals[i][0] > now:
                time.sleep(min(arrivals[i][0] - now, 0.0005))
                continue
            while i < len(arrivals) and arrivals[i][0] <= now:
                a, k = arrivals[i]
                f = filters[k]
                lag.append(time.perf_counter() - t0 - a)  # host: arrival to issue
                f.step(0.1)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(f.stream)
                done.append((a, k, ev))
                i += 1
        torch.cuda.synchronize()
    finally:
        gc.enable()
    wall = time.perf_counter() - t0
    lat = np.array([start.elapsed_time(ev) * 1e-3 - a for a, _, ev in done])
    updates = sum(int(admitted[k]["nu"]) for _, k, _ in done)
    last = max(start.elapsed_time(ev) for _, _, ev in done) * 1e-3
    for f in filters:
        f.close()
    return {
        "workload": f"serving: {n_streams} streams (sides 256/512/1024, 16 particles per cell), "
                    f"Poisson 10 Hz each, {budget_gb:.0f} GB admission",
        "arm": "plain: one stream, requests in arrival order" if plain else
               "concurrent: a CUDA stream per filter, requests of different streams overlap",
        "streams_admitted": len(admitted), "streams_rejected": rejected,
        "workspace_gb": used / 1e9, "seconds": seconds, "requests": len(done),
        "offered_particle_updates_per_s": sum(float(c["nu"]) * c["rate_hz"] for c in admitted),
        "served_particle_updates_per_s": updates / last,
        "updates": updates, "last_completion_s": last,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
        "issue_lag_ms": {"p99": float(np.percentile(lag, 99) * 1e3), "max": float(max(lag) * 1e3)},
        "wall_s": wall,
    }


def run_sessions(n_streams: int = 256, seconds: float = 3.0, budget_gb: float = 40.0, slots: int = 64,
                 mean_session_s: float = 1.0, connect_s: float = 1.5, seed: int = 7, cfgs: list = None,
                 keep: bool = False) -> dict:
    """Streams that come and go.  Stream k connects at a uniform time in [0, connect_s) and
    wants a session of Exp(mean_session_s) seconds; admitted (Admission: arrival order,
    budget_gb and `slots` streams at once), it gets a filter and a device grid, and its
    first request (which also captures the filter's CUDA graph) is issued at once; further
    requests (one frame each) follow by a Poisson process at its rate until its session ends
    (at `seconds` at the latest).  Once its session is over and its last frame has finished
    on the GPU, its filter is destroyed and its workspace freed, and waiting streams are
    admitted in its place.  Opening and closing filters run on a worker thread (the
    library's graph capture is thread-local), so the request loop never waits for them;
    each filter gets a CUDA stream of its own for its lifetime (torch's pooled streams are
    shared between filters, and no other filter's work may enter a stream while the
    worker captures a new filter's graph on it).
    With keep=True the result lists every served stream's frame count, grid and final
    cells, to be checked against the same stream run alone."""
    cfgs = scene.serving_stream_configs(n_streams) if cfgs is None else cfgs
    n = len(cfgs)
    rng = np.random.default_rng(seed)
    connect = np.sort(rng.uniform(0.0, connect_s, n))
    life = rng.exponential(mean_session_s, n)
    need = [stream_need(c) for c in cfgs]
    adm = Admission(budget_gb * 1e9, slots)
    todo, opened, closed = queue.Queue(), queue.Queue(), queue.Queue()
    # each stream's measurement grid, as its sensor would deliver it (made before the run)
    grids = [scene.random_measurement_grid(c["width"], c["height"], rng) for c in cfgs]

    failed = queue.Queue()  # an exception of the worker, re-raised by the request loop

    def worker():
        try:
            serve_jobs()
        except BaseException as e:  # noqa: BLE001 -- handed to the request loop
            failed.put(e)

    def serve_jobs():
        while True:
            job = todo.get()
            if job is None:
                return
            kind, k, obj = job
            if kind == "close":
                f, raw = obj
                f.close()  # waits for the stream, frees workspace and grid buffers
                _check(cudart.cudaStreamDestroy(raw)[0])
                del f, obj, job
                closed.put(k)
                continue
            ta = time.perf_counter()
            c = cfgs[k]
            err, raw = cudart.cudaStreamCreateWithFlags(cudart.cudaStreamNonBlocking)
            _check(err)
            f = DogFilter(scene.filter_params(c, seed=500 + k), stream=torch.cuda.ExternalStream(int(raw)))
            g = grids[k]
            f.set_measurement_grid(**{kk: torch.tensor(v, device="cuda") for kk, v in g.items()})
            f.step(0.1)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(f.stream)
            opened.put((k, f, raw, g, ev, obj, time.perf_counter() - ta))

    th = threading.Thread(target=worker, daemon=True)
    live, served, waits, done, first = {}, {}, [], [], []
    pending = 0  # admitted, not yet opened or not yet closed
    open_s, n_open, max_live = 0.0, 0, 0
    gc.collect()
    gc.disable()  # as in run(): no collection pass while requests are issued
    try:
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        torch.cuda.synchronize()
        th.start()
        t0 = time.perf_counter()
        ci = 0
        while True:
            if not failed.empty():
                raise RuntimeError("serving worker failed while opening or closing a filter") from failed.get()
            if not th.is_alive():
                raise RuntimeError("serving worker exited unexpectedly")
            now = time.perf_counter() - t0
            while ci < n and connect[ci] <= now:
                adm.request(ci, need[ci])
                ci += 1
            while not closed.empty():
                adm.release(closed.get())
                pending -= 1
            if now < seconds:
                for k in adm.admit():
                    waits.append(now - connect[k])
                    todo.put(("open", k, now))
                    pending += 1
            while not opened.empty():  # first frame issued by the worker at admission time
                k, f, raw, g, ev, t_req, dt = opened.get()
                pending -= 1
                open_s += dt
                n_open += 1
                nu = int(cfgs[k]["nu"])
                first.append((t_req, ev))
                done.append((t_req, nu, ev))
                live[k] = dict(f=f, raw=raw, grid_host=g if keep else None, t_end=min(t_req + life[k], seconds),
                               next=time.perf_counter() - t0 + rng.exponential(1.0 / cfgs[k]["rate_hz"]),
                               last=ev, frames=1, rate=cfgs[k]["rate_hz"], nu=nu)
            max_live = max(max_live, len(live))
            issued = False
            for k in list(live):
                s = live[k]
                now = time.perf_counter() - t0
                while s["next"] <= now and s["next"] < s["t_end"]:  # requests due
                    s["f"].step(0.1)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(s["f"].stream)
                    done.append((s["next"], s["nu"], ev))
                    s["last"] = ev
                    s["frames"] += 1
                    s["next"] += rng.exponential(1.0 / s["rate"])
                    issued = True
                if now >= s["t_end"] and s["last"].query():  # session over, last frame finished
                    served[k] = dict(frames=s["frames"])
                    if keep:
                        served[k].update(grid=s["grid_host"], cells=s["f"].cells(["m_occ", "m_free", "p_occ"]))
                    todo.put(("close", k, (s["f"], s["raw"])))
                    pending += 1
                    del live[k]
            if now >= seconds and not live and pending == 0:
                break
            if not issued:
                time.sleep(0.0002)
    finally:
        gc.enable()
    todo.put(None)
    th.join()
    torch.cuda.synchronize()
    t_first = {id(ev) for _, ev in first}
    lat = np.array([start.elapsed_time(ev) * 1e-3 - a for a, _, ev in done if id(ev) not in t_first])
    lat1 = np.array([start.elapsed_time(ev) * 1e-3 - a for a, ev in first])
    updates = sum(nu for _, nu, _ in done)
    last = max(start.elapsed_time(ev) for _, _, ev in done) * 1e-3
    w = np.array(waits)
    out = {
        "workload": f"serving sessions: {n} streams connecting over {connect_s:g} s, sessions "
                    f"Exp({mean_session_s:g} s), {budget_gb:.0f} GB and {slots} slots",
        "streams_served": len(served), "streams_never_admitted": n - len(served),
        "most_streams_at_once": max_live, "requests": len(done),
        "admitted_after_waiting": int((w > 0.01).sum()),
        "wait_s": {"p50": float(np.percentile(w, 50)), "max": float(w.max())},
        "open_ms_mean": open_s / max(n_open, 1) * 1e3,
        # admission to the end of the stream's first frame (filter set-up on the worker,
        # queued behind the other streams admitted at the same time, and graph capture)
        "first_frame_ms": {"p50": float(np.percentile(lat1, 50) * 1e3), "p99": float(np.percentile(lat1, 99) * 1e3)},
        "served_particle_updates_per_s": updates / last, "updates": updates,
        # the requests after each stream's first frame
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
    }
    if keep:
        out["served"] = served
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=256)
    ap.add_argument("--seconds", type=float, default=3.0)
    ap.add_argument("--budget-gb", type=float, default=None)
    ap.add_argument("--sessions", action="store_true", help="streams that come and go")
    ap.add_argument("--plain", action="store_true", help="one stream, requests in arrival order")
    args = ap.parse_args()
    if args.sessions:
        print(json.dumps(run_sessions(args.streams, args.seconds, args.budget_gb or 40.0)))
    else:
        print(json.dumps(run(args.streams, args.seconds, args.budget_gb or 120.0, plain=args.plain)))


if __name__ == "__main__":
    main()
