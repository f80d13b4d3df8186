"""Partition of the local problems (Section 3) across ranks, one GPU per rank.

The local problems are independent units: each rank solves a contiguous range of the leaf
list and nothing is exchanged on the data path (the caller gathers results, if it needs them,
off the hot path). Ranges are balanced by the expected work of a leaf, which is proportional
to its cell count s^2 (the number of steps to steady state varies far less with s than s^2).
"""
from __future__ import annotations

import numpy as np


def leaf_shard(sizes, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of this rank's leaves: contiguous, balanced by the sum of s^2.

    Rank r takes the leaves whose prefix work (the work of all leaves before and including
    it) lies in (r W / world, (r + 1) W / world], W the total work, so the ranges tile the
    list exactly once for any world size, and every rank's share differs from W / world by
    at most one leaf's work."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    s = np.asarray(sizes, dtype=np.int64)
    if s.ndim != 1:
        raise ValueError("sizes must be one-dimensional")
    n = int(s.size)
    if n == 0:
        return 0, 0
    prefix = np.cumsum(s * s)
    total = int(prefix[-1])

    def edge(r: int) -> int:
        # first leaf whose prefix work exceeds r W / world (integer arithmetic: exact)
        return int(np.searchsorted(prefix * world, r * total, side="right"))

    start = 0 if rank == 0 else edge(rank)
    stop = n if rank == world - 1 else edge(rank + 1)
    return start, stop
