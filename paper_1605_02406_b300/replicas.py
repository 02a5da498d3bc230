"""Independent filters across processes, one process per GPU (torchrun).

A single filter does not shard: N ranks run N replicas of it on their own seeds and only
the timing is combined.  Workloads made of many independent filters (the batched and the
serving workloads) are split instead: each filter is placed on one rank by its HBM need
(place_by_budget), computed identically on every rank, so the placement needs no message.

Whole-job throughput is the units all ranks processed divided by the slowest rank's time
(every rank is timed between the same two barriers).  The reductions work on any
torch.distributed backend: NCCL with CUDA tensors on the GPU, gloo with CPU tensors in the
tests.
"""
from __future__ import annotations

import os


def rank_env() -> tuple:
    """(world size, global rank, local rank) from the launcher's environment (1, 0, 0
    without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base: int, rank: int) -> int:
    """Seed of a rank's replica: independent random streams per rank."""
    return base + rank


def slowest(value: float, device="cpu") -> float:
    """The largest of the ranks' values (their elapsed times); the value itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds: float, device="cpu") -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling: every rank
    processes units_per_rank)."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    return world * units_per_rank / slowest(seconds, device)


def total(value: float, device="cpu") -> float:
    """Sum of the ranks' values (units processed); the value itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def place_by_budget(need: list, world: int, budget: float) -> list:
    """Rank of each independent filter (-1: rejected), given its HBM need in bytes and a
    budget per rank: filters in order, each to the rank with the fewest bytes placed so far
    among those it still fits (the lowest such rank on a tie).  With one rank this admits
    filters in order while they fit."""
    used = [0.0] * world
    out = []
    for b in need:
        best = -1
        for r in range(world):
            if used[r] + b <= budget and (best < 0 or used[r] < used[best]):
                best = r
        if best >= 0:
            used[best] += b
        out.append(best)
    return out
