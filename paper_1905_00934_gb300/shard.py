"""Slice sharding across ranks (one process per GPU).

Slices are independent ADMM problems (Sec. 3.3 per slice), so ranks reconstruct disjoint slices and
exchange nothing on the data path. Ranks take contiguous slice ranges balanced by a per-slice cost:
the iteration's work is dominated by R and R^T (Table 1), whose cost grows with the number of
projection-matrix weights, about n_views * n_bins * max(nx, ny) per basis.
"""
from __future__ import annotations

from typing import Sequence


def slice_cost(nx: int, ny: int, n_views: int, n_bins: int, iterations: int = 1) -> float:
    """Relative cost of reconstructing one slice: projector weights x iterations."""
    return float(n_views) * float(n_bins) * float(max(nx, ny)) * float(iterations)


def _fits(costs: Sequence[float], parts: int, cap: float) -> bool:
    used, load = 1, 0.0
    for c in costs:
        if c > cap:
            return False
        if load + c > cap:
            used += 1
            load = c
        else:
            load += c
    return used <= parts


def _greedy(costs: Sequence[float], cap: float) -> list[tuple[int, int]]:
    """Contiguous ranges filled in order up to `cap` each (the rule _fits counts)."""
    ranges, start, load = [], 0, 0.0
    for i, c in enumerate(costs):
        if load + c > cap and i > start:
            ranges.append((start, i))
            start, load = i, 0.0
        load += c
    ranges.append((start, len(costs)))
    return ranges


def partition(costs: Sequence[float], parts: int) -> list[tuple[int, int]]:
    """Splits slices 0..n-1 into `parts` contiguous ranges [lo, hi) minimising the largest range cost.

    Exact: feasibility is monotone in the capacity, so bisection over doubles finds the smallest
    feasible capacity to the last bit; the greedy ranges at that capacity have the optimal largest
    cost (a run sum, and no run sum lies between the optimum and that capacity). O(n) per step,
    about 64 steps. Ranges may be empty when there are fewer slices than parts.
    """
    if parts < 1:
        raise ValueError("parts must be >= 1")
    n = len(costs)
    if any(c < 0 for c in costs):
        raise ValueError("costs must be >= 0")
    if n == 0:
        return [(0, 0)] * parts
    # the bounds: the largest slice (may be infeasible) and the total, added in order as _fits adds
    # (Python's sum() of floats is compensated and can land one ulp below that running total)
    total = 0.0
    for c in costs:
        total += c
    lo, hi = max(costs), total
    if _fits(costs, parts, lo):
        hi = lo
    while True:
        mid = lo + (hi - lo) / 2
        if mid <= lo or mid >= hi:
            break
        if _fits(costs, parts, mid):
            hi = mid
        else:
            lo = mid
    ranges = _greedy(costs, hi)
    while len(ranges) < parts:
        ranges.append((n, n))
    return ranges


def rank_slices(costs: Sequence[float], rank: int, world_size: int) -> range:
    """The slice indices rank `rank` of `world_size` reconstructs."""
    lo, hi = partition(costs, world_size)[rank]
    return range(lo, hi)


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's); `value` itself
    without an initialised process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
