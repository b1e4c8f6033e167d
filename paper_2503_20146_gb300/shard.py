"""Sharding of independent projections across ranks (one GPU per rank).

Every projection is its own PWF problem and the diffuser is read-only, so a
series splits across ranks with no exchange during the iterations: each rank
builds one plan per size class over its share and runs pwf_solve; results are
gathered once at the end. Shares are balanced by cost, the pixels of a
projection times its number of source modes (the passes are linear in both).
"""
from __future__ import annotations

import heapq
from typing import Sequence


def projection_cost(ny: int, nx: int, n_modes: int = 0) -> int:
    return int(ny) * int(nx) * max(1, int(n_modes))


def shard_projections(shapes: Sequence[tuple], world: int, rank: int) -> list:
    """Indices of the projections rank `rank` of `world` should solve.

    shapes: per projection (ny, nx) or (ny, nx, n_modes). Greedy
    longest-processing-time assignment: projections in decreasing cost, each to
    the least-loaded rank (ties to the lower rank), so every rank's load is
    within one projection's cost of the mean. Indices come back sorted.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    costs = [projection_cost(*s) for s in shapes]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return sorted(mine)


def rank_loads(shapes: Sequence[tuple], world: int) -> list:
    """Total cost assigned to each rank by shard_projections."""
    return [sum(projection_cost(*shapes[i]) for i in shard_projections(shapes, world, r)) for r in range(world)]
