"""Replica bookkeeping for runs on several GPUs (one process per GPU).

The matcher's units of work (rectified pairs, serving frames) are
independent, so they shard across ranks as whole pairs with no exchange
step: no collective touches the data.  The one collective is the timing
reduction: the job takes as long as its slowest rank, and its rate counts
the units of every rank.  Works with the nccl backend (CUDA tensors) and
gloo (CPU tensors).
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(RANK, LOCAL_RANK, WORLD_SIZE) as torch.distributed.run exports them."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(n_items: int, rank: int, world: int) -> range:
    """Whole items of rank `rank`: round-robin, disjoint, covering 0..n_items-1."""
    if not 0 <= rank < world:
        raise ValueError("rank outside the world")
    return range(rank, n_items, world)


def _reduce(value: float, op: str, dist, device) -> float:
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op))
    return float(t.item())


def max_over_ranks(value: float, dist=None, device=None) -> float:
    return _reduce(value, "MAX", dist, device)


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    return _reduce(value, "SUM", dist, device)


def job_rate(units: float, seconds: float, dist=None, device=None) -> tuple[float, float, float]:
    """(units of all ranks, the slowest rank's seconds, units per second)."""
    total = sum_over_ranks(units, dist, device)
    slowest = max_over_ranks(seconds, dist, device)
    return total, slowest, total / slowest
