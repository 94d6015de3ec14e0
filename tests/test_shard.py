"""Range sharding across ranks: cost balance and a world-size-2 gloo run.

The multi-GPU form of the search gives each rank a contiguous sub-range with
equal cumulative cost sum p and concatenates the hit lists on the host.  Here
the ranks are CPU processes on the gloo backend and the per-rank search is the
oracle's (sieve, then B_{p-3} and E_{p-3} mod p by their definitions), so the
host logic -- split, per-rank ranges, gather, merge -- is exercised without a
GPU.
"""
import os
import socket

import numpy as np
import pytest

from paper_2101_11157_gb300 import shard


def test_split_covers_range_and_is_monotone():
    for lo, hi, n in [(5, 50_000, 1), (5, 50_000, 2), (1_000_000, 2_000_000, 7),
                      (10**11 - 10**4, 10**11, 8), (100, 101, 4), (7, 7, 3)]:
        b = shard.split_range(lo, hi, n)
        assert len(b) == n + 1 and b[0] == lo and b[-1] == hi
        assert all(x <= y for x, y in zip(b, b[1:]))


def test_split_balances_sum_of_primes(orc):
    # cost of a shard = sum of its primes (work per prime is proportional to p)
    lo, hi, n = 1_000, 30_000_000, 4
    b = shard.split_range(lo, hi, n)
    pr = orc.sieve(lo, hi).astype(np.float64)
    sums = [pr[(pr >= b[k]) & (pr < b[k + 1])].sum() for k in range(n)]
    assert max(sums) / min(sums) < 1.01
    # an even split by integers would be badly unbalanced here
    even = [lo + (hi - lo) * k // n for k in range(n + 1)]
    sums_even = [pr[(pr >= even[k]) & (pr < even[k + 1])].sum() for k in range(n)]
    assert max(sums_even) / min(sums_even) > 3


def test_shard_of_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.shard_of(5, 100, 2, 2)
    with pytest.raises(ValueError):
        shard.split_range(5, 100, 0)


def _oracle_search(a, b):
    from oracle import oracle as O
    a = max(a, 5)
    if b <= a:
        return []
    hits = []
    for p in O.sieve(a, b).tolist():
        kind = (1 if O.bernoulli_def(p - 3, p) == 0 else 0) | (2 if O.euler_def(p - 3, p) == 0 else 0)
        if kind:
            hits.append((p, kind))
    return hits


def _worker(rank, world, port, lo, hi, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        a, b = shard.shard_of(lo, hi, rank, world)
        hits = shard.sharded_search(lo, hi, search=_oracle_search)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{a} {b}\n")
            f.write(" ".join(f"{p}:{k}" for p, k in hits) + "\n")
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_search_gloo_world2(orc, tmp_path):
    import torch.multiprocessing as mp
    lo, hi, world = 5, 1_000, 2
    mp.spawn(_worker, args=(world, _free_port(), lo, hi, str(tmp_path)), nprocs=world, join=True)
    ranges, results = [], []
    for r in range(world):
        with open(tmp_path / f"rank{r}.txt") as f:
            a, b = map(int, f.readline().split())
            line = f.readline().split()
        ranges.append((a, b))
        results.append([tuple(map(int, t.split(":"))) for t in line])
    # the sub-ranges tile [lo, hi) and every rank returns the same merged list
    assert ranges[0][0] == lo and ranges[-1][1] == hi and ranges[0][1] == ranges[1][0]
    assert results[0] == results[1]
    # ... which equals the unsharded search: B hit 16843 is above 1000, so the
    # hits below 1000 are the Vandiver primes 149 and 241 (Sec. 1)
    assert results[0] == _oracle_search(lo, hi) == [(149, 2), (241, 2)]


@pytest.mark.gpu
def test_shards_on_one_gpu_union_equals_whole():
    # every shard searched on this GPU; the union equals the unsharded search,
    # hits and residues alike (the window holds the Vandiver prime 1062232319)
    import torch
    from paper_2101_11157_gb300 import api
    lo, hi = 1_062_200_000, 1_062_300_000
    whole, pr, rb, re = api.search(lo, hi, near=50, with_residues=True)
    bounds = shard.split_range(lo, hi, 4)
    parts, res = [], []
    for a, b in zip(bounds, bounds[1:]):
        h, p, x, y = api.search(a, b, near=50, with_residues=True)
        parts.append(h)
        res.append((p, x, y))
    assert shard.merge_hits(parts) == sorted(whole)
    cat = [torch.cat([r[i] for r in res]) for i in range(3)]
    assert torch.equal(cat[0], pr) and torch.equal(cat[1], rb) and torch.equal(cat[2], re)
    assert [p for p, _ in whole] == [1_062_232_319]
