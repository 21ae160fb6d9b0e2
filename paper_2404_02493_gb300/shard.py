"""A batch of independent Helmholtz instances over several ranks (one process
per GPU).

The instances of a batch share nothing, so a batch shards without any
collective on the data path: rank r sets up a handle with a contiguous range
of the instances and solves them on its own GPU.  The ranges are balanced by
the work of an instance (its fine grid points).  Only the per-instance results
travel, once, to the host of every rank (`gather_to_host`), plus whatever
timing reductions a benchmark adds.
"""
from __future__ import annotations

from typing import Sequence


def shard_ranges(work: Sequence[float], world: int) -> list[tuple[int, int]]:
    """Contiguous half-open ranges [lo, hi) of the instances, one per rank,
    in rank order, covering every instance once.  The boundary after rank r
    takes every instance whose midpoint (in cumulative work) lies at or below
    the fraction (r + 1) / world of the total, so each boundary is within half
    an instance of an even split; a rank can get an empty range when there
    are fewer instances than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if any(w < 0 for w in work):
        raise ValueError("work must be non-negative")
    total = float(sum(work))
    out = []
    lo, acc, i = 0, 0.0, 0
    for r in range(world):
        if r == world - 1:
            hi = len(work)
        else:
            target = total * (r + 1) / world
            hi = lo
            while hi < len(work) and acc + work[hi] / 2 <= target:
                acc += work[hi]
                hi += 1
        out.append((lo, hi))
        lo = hi
    return out


def my_shard(work: Sequence[float], rank: int, world: int) -> range:
    lo, hi = shard_ranges(work, world)[rank]
    return range(lo, hi)


def gather_to_host(local: dict, world: int) -> dict:
    """Merge the per-instance results {instance index: value} of all ranks
    (host objects) on every rank; with one rank the input is returned."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local)
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"instance {k} solved on two ranks")
            merged[k] = v
    return merged
