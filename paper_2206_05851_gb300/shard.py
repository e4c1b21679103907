"""Multi-GPU form of the method: weak scaling over independent chain sets.

Chains (and their replicas) never exchange data, so N ranks - one process per
GPU - each integrate a chain set of the workload's shape with their own
Philox key and their own initial coils; there is no collective on the data
path. The timed region is bracketed by barriers and its length is the
maximum over ranks; the whole-job throughput is the work of all ranks over
that time. These helpers hold that host logic so that it runs unchanged
under NCCL (one GPU per rank) and gloo (CPU tests).
"""
from __future__ import annotations

from typing import Optional, Tuple

RANK_SEED_STRIDE = 1000


def rank_keys(seed: int, init_seed: int, rank: int) -> Tuple[int, int]:
    """(Philox key, initial-coil seed) of a rank's chain set: rank 0 keeps
    the workload's own, rank r shifts the key by r * RANK_SEED_STRIDE (a
    disjoint noise stream, since the key selects the Philox permutation) and
    the coil seed by r."""
    if rank < 0:
        raise ValueError("rank must be >= 0")
    return seed + RANK_SEED_STRIDE * rank, init_seed + rank


def max_over_ranks(value: float, dist=None, device: Optional[str] = None) -> float:
    """Maximum of a per-rank float over the process group (the value itself
    with no group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_max_s: float) -> float:
    """Units of all ranks per second of the slowest rank's time."""
    if t_max_s <= 0:
        raise ValueError("time must be > 0")
    return units_per_rank * world / t_max_s
