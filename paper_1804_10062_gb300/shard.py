"""Assignment of independent sort units (batched segments, served requests)
to ranks: one process per GPU, no data-path collective.

The plain sort of one array does not shard (its rounds form a serial chain on
one shared array), so it runs as replicas.  Batched segments and served
requests are independent; they are spread over ranks by LPT (longest
processing time first: units in decreasing cost order, each to the rank with
the least cost so far), with cost n log2 n, the comparison-count order of
QuickMergesort.
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def unit_cost(n: int) -> float:
    return float(n) * math.log2(n) if n > 1 else 0.0


def lpt_assign(lengths, world_size: int):
    """Returns a list of index arrays, one per rank (ascending indices)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    lengths = np.asarray(lengths, dtype=np.int64)
    cost = np.where(lengths > 1, lengths * np.log2(np.maximum(lengths, 2)), 0.0)
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, r) for r in range(world_size)]
    out = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(int(i))
        heapq.heappush(heap, (load + float(cost[i]), r))
    return [np.array(sorted(v), dtype=np.int64) for v in out]


def rank_loads(lengths, assignment):
    lengths = np.asarray(lengths, dtype=np.int64)
    return [sum(unit_cost(int(lengths[i])) for i in a) for a in assignment]


def local_segments(offsets, assignment_for_rank):
    """Offsets of this rank's segments packed contiguously, and for each
    local segment its (begin, end) in the global array."""
    offsets = np.asarray(offsets, dtype=np.uint64)
    b = offsets[assignment_for_rank]
    e = offsets[assignment_for_rank + 1]
    lens = (e - b).astype(np.uint64)
    loc = np.zeros(len(lens) + 1, dtype=np.uint64)
    np.cumsum(lens, out=loc[1:])
    return loc, b, e
