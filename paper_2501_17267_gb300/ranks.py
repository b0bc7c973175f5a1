"""Weak scaling across GPUs: the host logic of a multi-rank run.

The method's units are independent (instances; SA replicas; serving requests), so N
ranks -- one process per GPU -- each solve their own share with no collective on the
data path.  The only collective is the timing: every rank times its own step and the
job's time is the slowest rank's.  The whole-job rate is the units of all ranks over
that time.
"""
from __future__ import annotations


def rank_units(rank: int, per_rank: int):
    """Global indices of the units (instances) of `rank` when every rank takes
    `per_rank`: disjoint across ranks, the same on every run."""
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks of the default process group (x itself without one).
    device: where the reduction tensor lives (a CUDA device for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: float, world: int, steps: int, max_ms: float) -> float:
    """Whole-job rate: every rank's units of every step over the slowest rank's time."""
    return units_per_rank_step * world * steps / (max_ms / 1000.0)
