"""Rank bookkeeping for running the particle advance as independent replicas.

Every box holds one GPU, and the per-step advance of independent particle sets
needs no exchange: N processes each advance their own particles (own seed)
against their own copy of the fields.  The only cross-rank traffic is the
timing reduction (the slowest rank sets the job's time) and barriers around the
timed region.  Works with the nccl backend on GPUs and gloo on CPUs.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s particle set: distinct per rank, equal to `seed`
    on rank 0 so that a one-rank run is the single-GPU workload."""
    return int(seed) + 1000003 * int(rank)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest `value` over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * steps * world / seconds
