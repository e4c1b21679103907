"""Multi-GPU form of the method: one workload split over ranks.

The parent chains of a workload, each with its replica set, are independent
simulations (Sec. II: the replicas are quasi-independent simulations of the
halted parent, and chains never interact), so the chain list is split into
contiguous ranges, one per rank (one process per GPU), with no exchange
during the integration. Each rank's context takes its range's first global
chain index as ``chain_id_base``, so that its chains draw the noise of the
whole workload: the union of the ranks' results is, bit for bit, the result
of the whole workload in one context. The ranges are balanced by the cost of
a chain, N (R + 1) slot-beads a step (parent and replicas).

The only collectives come after the integration: the event lists are
gathered (each rank's list is in (chain, spring, criterion, kind) order and
the ranges are in chain order, so the concatenation in rank order is the
whole workload's list) and the per-rank histograms and survival terms are
summed. The timed region is bracketed by barriers and its length is the
maximum over ranks; the whole-job throughput is the work of all ranks over
that time. These helpers hold that host logic so that it runs unchanged
under NCCL (one GPU per rank) and gloo (CPU tests).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def chain_cost(chain) -> int:
    """Slot-bead updates of one integration step: N (R + 1)."""
    return int(chain.n_beads) * (int(chain.n_replicas) + 1)


def partition(costs: Sequence[float], world: int) -> List[Tuple[int, int]]:
    """Contiguous [begin, end) chain ranges, one per rank, that split the
    prefix sum of `costs` as evenly as a contiguous split allows: rank r's
    range ends at the chain boundary nearest to (r + 1) / world of the total
    cost, and every rank gets at least one chain while chains remain."""
    n = len(costs)
    if world < 1:
        raise ValueError("world must be >= 1")
    if n < world:
        raise ValueError(f"{n} chains cannot be split over {world} ranks")
    c = np.concatenate([[0.0], np.cumsum(np.asarray(costs, dtype=np.float64))])
    total = c[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(c, target))            # first prefix >= target
        if k > 0 and target - c[k - 1] <= c[k] - target:
            k -= 1
        lo = bounds[-1] + 1                            # at least one chain for rank r - 1
        hi = n - (world - r)                           # and one for each later rank
        bounds.append(min(max(k, lo), hi))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def rank_range(chains: Sequence, rank: int, world: int) -> Tuple[int, int]:
    """This rank's [begin, end) range of the workload's chains."""
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return partition([chain_cost(ch) for ch in chains], world)[rank]


def rank_share(chains: Sequence, pos0: np.ndarray, rank: int, world: int):
    """(chains, initial positions [sum N][3], chain_id_base) of this rank's
    range; pos0 holds the whole workload's positions in chain order."""
    begin, end = rank_range(chains, rank, world)
    offs = np.concatenate([[0], np.cumsum([ch.n_beads for ch in chains])])
    return list(chains[begin:end]), np.asarray(pos0)[offs[begin]:offs[end]], begin


def globalize_events(events: np.ndarray, chain_id_base: int) -> np.ndarray:
    """A rank's event list (structured array with a 'chain' field, chain
    indices local to the rank's context) with whole-workload chain indices."""
    out = np.array(events, copy=True)
    out["chain"] += chain_id_base
    return out


def gather_events(events: np.ndarray, dist=None) -> Optional[np.ndarray]:
    """Concatenation in rank order of every rank's (globalized) event list,
    on rank 0 (None elsewhere); the list itself with no group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return events
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, events)
    return np.concatenate(parts) if dist.get_rank() == 0 else None


def gather_rows(rows: np.ndarray, dist=None) -> Optional[np.ndarray]:
    """Per-chain (or per-spring) arrays of the ranks joined along their last
    axis in rank order (e.g. log-survival [n_chains][3] transposed, RSF
    history [W][M_rank]); on rank 0, None elsewhere."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return rows
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, np.asarray(rows))
    return np.concatenate(parts, axis=-1) if dist.get_rank() == 0 else None


def sum_counts(counts: np.ndarray, dist=None, device: Optional[str] = None) -> np.ndarray:
    """Element-wise sum over ranks of a count or histogram array."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return np.asarray(counts)
    import torch
    t = torch.as_tensor(np.asarray(counts, dtype=np.float64), device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def max_over_ranks(value: float, dist=None, device: Optional[str] = None) -> float:
    """Maximum of a per-rank float over the process group (the value itself
    with no group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_all_ranks: float, t_max_s: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    if t_max_s <= 0:
        raise ValueError("time must be > 0")
    return units_all_ranks / t_max_s
