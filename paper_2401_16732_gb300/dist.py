"""Multi-rank bookkeeping of the throughput measurement.

The path shards without any data exchange (each rank convolves its own
images), so the only collective is this one: the slowest rank's time and the
whole-job throughput.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity when not distributed)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_this_rank: float, device=None) -> tuple[float, float]:
    """(units of all ranks / slowest rank's seconds, slowest seconds); every
    rank processes the same number of units (weak scaling)."""
    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    slowest = max_over_ranks(seconds_this_rank, device)
    return world * units_per_rank / slowest, slowest
