"""Partition of a batch of independent instances over ranks.

Instances never exchange data, so sharding is an assignment problem: greedy
longest-first (LPT) assignment of instances to the least-loaded rank, the
load of an instance taken as n (l + 1)^2 (its sweeps do O(l^2) work per row
and their time is dominated by the longest instances).  Host-side only.
"""
from __future__ import annotations

import heapq


def instance_cost(n: int, l: int) -> int:
    return int(n) * (int(l) + 1) ** 2


def partition(ns, ls, world: int):
    """Returns, for each rank, the sorted list of instance indices it owns."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(ns)), key=lambda i: (-instance_cost(ns[i], ls[i]), i))
    heap = [(0, r) for r in range(world)]
    owned = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        owned[r].append(i)
        heapq.heappush(heap, (load + instance_cost(ns[i], ls[i]), r))
    return [sorted(o) for o in owned]


def loads(ns, ls, parts):
    return [sum(instance_cost(ns[i], ls[i]) for i in p) for p in parts]
