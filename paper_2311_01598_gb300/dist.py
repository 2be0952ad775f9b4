"""Multi-GPU plumbing for key switching: data parallelism over ciphertexts.

Independent key switches shard across ranks with no collective on the data
path (each rank owns its jobs, keys and outputs); the only collectives are
the benchmark's barrier and the max-over-ranks of its timings.  One process
per GPU (torchrun), NCCL on GPUs, gloo on CPU (tests).
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world: int):
    """Contiguous block of items owned by rank (sizes differ by at most one)."""
    n = len(items)
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return items[lo:hi]


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of a value over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank, seconds_per_rank, device=None) -> float:
    """Whole-job rate: units of all ranks over the slowest rank's time."""
    return sum_over_ranks(units_per_rank, device) / max_over_ranks(seconds_per_rank, device)
