"""Instance partition of one batch across ranks (one process per GPU).

Batched and served solves shard by instance: the instances are independent, so
a rank solves its share with no collective in the data path.  The share of
each rank comes from a greedy longest-processing-time partition on a work
estimate per instance (the nonzeros one PDHG step streams), which every rank
computes identically from the same instance list, so no list is exchanged.

Host logic only; the solves themselves run in the CUDA library.
"""
from __future__ import annotations

import heapq


def work_estimate(qp, diagonal_q: bool | None = None) -> int:
    """Nonzeros one PDHG step streams: A x and A^T y, plus Q products of the
    inner solver when Q is not diagonal (about four per step), plus the vectors."""
    nz_a = int(qp.A.nnz)
    q = getattr(qp, "Q", None)
    nz_q = int(q.nnz) if q is not None else 0
    if diagonal_q is None:
        diagonal_q = q is None or nz_q <= qp.n
    return 2 * nz_a + (0 if diagonal_q else 4 * nz_q) + int(qp.n) + int(qp.m)


def partition(weights, world: int):
    """Split instance indices 0..len(weights)-1 into ``world`` lists.

    Greedy LPT: instances in decreasing weight (ties by index) each go to the
    rank with the least assigned weight so far (ties by rank).  Deterministic,
    every index appears in exactly one list, each list is in increasing index
    order, and the largest load exceeds the smallest by at most the largest
    single weight."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + weights[i], r))
    return [sorted(p) for p in parts]


def loads(weights, parts):
    """Assigned weight per rank."""
    return [sum(weights[i] for i in p) for p in parts]
