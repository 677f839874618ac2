"""Event sharding over GPUs, one process per GPU: cost-balanced contiguous ranges
of one event list, and the host-side gather of the per-event results.

Events are independent integrals (Sec. 2: every integration point is
independent, and each event's integral uses only its own points), so the ranks
exchange nothing on the data path: each rank integrates its own contiguous
range of the list with event ids starting at the range's first index (the
Philox streams, and so the results, are those of one process integrating the
whole list), and only the per-event results (p-hat, error, points used, status;
32 bytes per event) are gathered on the host at the end.

Cost model of an event: integration dimensions x jet permutations x points per
(event, permutation) item -- the integrand evaluations it needs, weighted by
the width of each evaluation's map. The ranges minimise the largest rank's cost.
"""
from __future__ import annotations

import numpy as np

from . import synth


def event_cost(kinds, points_per_item):
    """Cost of each event: dims x permutations x points per item (int64).
    kinds: process kind per event; points_per_item: scalar or per event."""
    kinds = np.asarray(kinds, dtype=np.int64)
    dims = np.array([synth.DIMS[int(k)] for k in range(max(synth.DIMS) + 1)], dtype=np.int64)
    nperm = np.array([synth.NPERM[int(k)] for k in range(max(synth.NPERM) + 1)], dtype=np.int64)
    pts = np.broadcast_to(np.asarray(points_per_item, dtype=np.int64), kinds.shape)
    return dims[kinds] * nperm[kinds] * pts


def _greedy(cum, limit, world):
    """Contiguous ranges, each filled up to `limit`; None if more than `world` are
    needed. cum: inclusive prefix sums of the costs."""
    n = len(cum)
    bounds = [0]
    start = 0
    base = 0
    while start < n:
        stop = int(np.searchsorted(cum, base + limit, side="right"))
        if stop == start:          # one event alone exceeds the limit
            return None
        bounds.append(stop)
        if len(bounds) - 1 > world:
            return None
        base = int(cum[stop - 1])
        start = stop
    while len(bounds) - 1 < world:  # empty ranges for surplus ranks
        bounds.append(n)
    return [(bounds[i], bounds[i + 1]) for i in range(world)]


def balanced_ranges(costs, world):
    """Split events 0..n-1 into `world` contiguous ranges (start, stop) whose
    largest total cost is the smallest possible (binary search on that cost with
    greedy filling). Ranges may be empty when there are fewer events than ranks."""
    costs = np.asarray(costs, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if costs.ndim != 1 or np.any(costs < 0):
        raise ValueError("costs must be a 1-D array of non-negative integers")
    n = len(costs)
    if n == 0:
        return [(0, 0)] * world
    cum = np.cumsum(costs)
    lo, hi = int(costs.max()), int(cum[-1])
    while lo < hi:
        mid = (lo + hi) // 2
        if _greedy(cum, mid, world) is None:
            lo = mid + 1
        else:
            hi = mid
    return _greedy(cum, lo, world)


def my_range(costs, rank, world):
    """This rank's (start, stop)."""
    return balanced_ranges(costs, world)[rank]


def gather_results(results, start, stop, n_events, world, group=None, dst=0):
    """Gather per-event result arrays of all ranks on rank `dst` (host side).
    results: dict name -> array of this rank's stop - start events. Returns the dict
    of full-length arrays on dst and None elsewhere. Needs torch.distributed
    initialised when world > 1."""
    local = {k: np.asarray(v) for k, v in results.items()}
    for k, v in local.items():
        if len(v) != stop - start:
            raise ValueError(f"{k}: {len(v)} entries for the range [{start}, {stop})")
    if world == 1:
        return local if n_events == stop - start and start == 0 else _place([(start, stop, local)], n_events)
    import torch.distributed as dist
    rank = dist.get_rank(group)
    parts = [None] * world if rank == dst else None
    dist.gather_object((start, stop, local), parts, dst=dst, group=group)
    if rank != dst:
        return None
    return _place(parts, n_events)


def _place(parts, n_events):
    out = {}
    covered = np.zeros(n_events, dtype=bool)
    for start, stop, arrs in parts:
        if covered[start:stop].any():
            raise ValueError("overlapping ranges")
        covered[start:stop] = True
        for k, v in arrs.items():
            if k not in out:
                out[k] = np.zeros((n_events,) + v.shape[1:], dtype=v.dtype)
            out[k][start:stop] = v
    if not covered.all():
        raise ValueError("the ranges do not cover every event")
    return out
