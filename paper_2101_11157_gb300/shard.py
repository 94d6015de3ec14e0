"""Range sharding of a search across ranks (one process per GPU).

Primes are independent, so a search over [lo, hi) splits into contiguous
sub-ranges, one per rank, with no exchange on the data path; each rank runs
the whole path (sieve, residues, flags) on its own sub-range and the hit
lists are concatenated on the host afterwards.

The work of one prime is proportional to p: the congruences of Sec. 3 and
Sec. 5 sum over fixed fractions of 0 < s < p (BB30 about 227p/6480 terms, EE33
about 27p/512).  Splitting by the number of integers would load the upper
ranks more, so the split balances the cumulative cost sum_{lo <= p < b} p.
With the prime density 1/ln x that cost is close to the integral of x / ln x,
which the split evaluates by composite Simpson quadrature and inverts by
bisection on integers.
"""
from __future__ import annotations

import math

import numpy as np

_SIMPSON_PANELS = 256


def cost(a: float, b: float) -> float:
    """Approximate sum of p over the primes of [a, b): integral of x / ln x."""
    a = max(float(a), 3.0)
    b = float(b)
    if b <= a:
        return 0.0
    x = np.linspace(a, b, 2 * _SIMPSON_PANELS + 1)
    f = x / np.log(x)
    h = (b - a) / (2 * _SIMPSON_PANELS)
    return float(h / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum()))


def split_range(lo: int, hi: int, n: int) -> list[int]:
    """Boundaries lo = b_0 <= b_1 <= ... <= b_n = hi with equal estimated cost
    in each [b_k, b_{k+1})."""
    lo, hi, n = int(lo), int(hi), int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    if hi < lo:
        raise ValueError("hi < lo")
    total = cost(lo, hi)
    bounds = [lo]
    for k in range(1, n):
        target = total * k / n
        a, b = bounds[-1], hi
        while a < b:  # smallest integer m with cost(lo, m) >= target
            m = (a + b) // 2
            if cost(lo, m) < target:
                a = m + 1
            else:
                b = m
        bounds.append(a)
    bounds.append(hi)
    return bounds


def shard_of(lo: int, hi: int, rank: int, world: int) -> tuple[int, int]:
    """The sub-range [a, b) that rank `rank` of `world` searches."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    b = split_range(lo, hi, world)
    return b[rank], b[rank + 1]


def merge_hits(parts) -> list[tuple[int, int]]:
    """Concatenate per-rank hit lists [(p, kind), ...] in ascending p."""
    out = [tuple(int(v) for v in h) for part in parts for h in part]
    out.sort()
    return out


def sharded_search(lo: int, hi: int, search=None, group=None):
    """Search [lo, hi) across the ranks of the initialised process group.

    Every rank calls this with the same (lo, hi); each searches its own
    cost-balanced sub-range with `search(a, b) -> [(p, kind), ...]` (by
    default the library's zero-residue search on this rank's GPU) and all
    ranks return the merged hit list.  Without an initialised process group
    the whole range is searched locally.
    """
    import torch.distributed as dist

    if search is None:
        from . import api

        def search(a, b):
            if b <= max(a, 5):
                return []
            return [(int(p), int(k)) for p, k in api.search(max(a, 5), b)]
    if not (dist.is_available() and dist.is_initialized()):
        return merge_hits([search(lo, hi)])
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a, b = shard_of(lo, hi, rank, world)
    local = search(a, b)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    return merge_hits(parts)


def expected_share(lo: int, hi: int, world: int) -> float:
    """Ideal fraction of the total cost per rank (1 / world)."""
    return 1.0 / world if world > 0 and hi > lo else math.nan
