"""Target sharding of one cluster across ranks (host-side logic).

The pair sums shard by target: rank r owns a contiguous range of star slots
and computes their accelerations against every source; the sources' O(N)
state is all-gathered before the pair passes and the hole's per-star terms
are all-reduced after them.  This module holds the ownership arithmetic and
the gather/reduce order; the pool this library runs on has one GPU per box,
so the multi-GPU data path itself is not built (bench.py runs replicas).
"""
from __future__ import annotations


def shard_ranges(n_bodies: int, world: int, align: int = 256) -> list[tuple[int, int]]:
    """Contiguous [start, stop) ranges of star bodies (1..n_bodies-1) per rank.

    Ranges are multiples of `align` stars except the last, so each rank's
    targets fill whole thread blocks; ranks beyond the work get empty ranges.
    """
    if n_bodies < 2 or world < 1:
        raise ValueError("need n_bodies >= 2 and world >= 1")
    ns = n_bodies - 1
    blocks = (ns + align - 1) // align
    per, extra = divmod(blocks, world)
    out, b = [], 0
    for r in range(world):
        nb = per + (1 if r < extra else 0)
        start = 1 + b * align
        stop = min(n_bodies, 1 + (b + nb) * align)
        out.append((start, max(start, stop)) if start < n_bodies else (n_bodies, n_bodies))
        b += nb
    return out


def owner_of(body: int, ranges: list[tuple[int, int]]) -> int:
    """Rank that owns star `body` (the hole, body 0, is replicated: rank 0)."""
    if body == 0:
        return 0
    for r, (a, b) in enumerate(ranges):
        if a <= body < b:
            return r
    raise ValueError(f"body {body} outside every range")
