"""Independent filter replicas, one process per GPU (torchrun): the filter itself does not
shard, so N ranks run N replicas on their own seeds and only the timing is combined.

Whole-job throughput is the units all ranks processed divided by the slowest rank's time
(every rank is timed between the same two barriers).  The reduction works on any
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
