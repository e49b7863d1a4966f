"""Assignment of independent units to ranks for the multi-GPU mode.

A single solve does not shard (the ML-cycle, the line search and the CD chain
are sequential).  Batched work does: each instance with its lambda path is an
independent unit, so the units are split over the ranks and every rank solves
its own share with no collective on the data path.  The split is the
longest-processing-time greedy rule: units in decreasing cost, each to the
rank with the least assigned cost so far (ties to the lowest rank).  Its
largest load is at most the average load plus the largest unit's cost, and at
most 4/3 of the optimum (Graham's bound for this rule).  Serving streams are
routed the same way, online: request k goes to the rank with the least
modelled work assigned before it (route_stream).
"""
from __future__ import annotations

import heapq
from typing import List, Sequence

# Cost model of one unit of dimension n, in units of a small solve: the dense
# factorisations grow as n^3, and a solve of n <= 512 is bound by its fixed
# launch and synchronisation latency (about the same time for any n up to 512).
_SMALL_N = 512.0


def unit_cost(n: int, solves: int = 1) -> float:
    """Relative time of `solves` solves (a lambda path) of dimension n."""
    return solves * (1.0 + (float(n) / _SMALL_N) ** 3)


def balanced_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of `costs` per rank (each list ascending).  Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if any(not (c >= 0.0) for c in costs):
        raise ValueError("costs must be non-negative numbers")
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + costs[k], r))
    return [sorted(ks) for ks in out]


def route_stream(costs: Sequence[float], world: int) -> List[int]:
    """Rank of each request of a stream, in arrival order: each request goes to
    the rank with the least modelled work assigned so far (ties to the lowest
    rank).  Online (no look-ahead), deterministic, and independent of timing,
    so every rank can compute the whole routing from the trace alone."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if any(not (c >= 0.0) for c in costs):
        raise ValueError("costs must be non-negative numbers")
    heap = [(0.0, r) for r in range(world)]
    out = []
    for c in costs:
        load, r = heapq.heappop(heap)
        out.append(r)
        heapq.heappush(heap, (load + c, r))
    return out
