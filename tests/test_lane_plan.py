"""Host-side model of the lane-chain planner (wv_residue.cu, k_lane_chains ..
k_chain_scatter): how many pieces a plan makes and where they go.

Each (prime, sum) of cnt terms becomes ceil(cnt / L) pieces, with L the
larger of a floor and the path's terms over the pieces wanted; the pieces are
sorted by class and length bin and every class is padded to whole warps.
The library sizes its buffers from a bound on the piece count (segments +
pieces wanted, or for a serving plan segments + terms / L from an upper bound
on the terms); these tests check that bound and the sort's invariants on
the library's own congruence rows, with the library's own interval
endpoints (wv_count_terms for the totals)."""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_2101_11157_gb300 import wv

SMS = 152
LANES = (768, 512)        # resident threads per SM: 32-bit kernel, 64-bit kernel
LMIN = (4096, 16384)      # shortest chain per path
ROUNDS, ROUNDS_EPOCH, LMAX_EPOCH = 16, 4, 1 << 17  # serving cap: the piece_log2 default


def _rows(cid):
    n = wv.wv_congruence_info(cid)[2]
    out = []
    for r in range(n):
        c = ctypes.c_int64()
        v = [ctypes.c_uint32() for _ in range(4)]
        wv.load().wv_congruence_row(cid, r, ctypes.byref(c), *[ctypes.byref(x) for x in v])
        out.append(tuple(x.value for x in v))
    return out


def _segments(primes, cb, ce):
    rows = [(w, 0) for w in _rows(cb)] + [(w, 1) for w in _rows(ce)]
    segs = []
    for p in sorted(int(x) for x in primes):
        for (xn, xd, yn, yd), kind in rows:
            lo = xn * p // xd + 1
            hi = yn * p // yd + 1
            segs.append((p, kind, max(0, hi - lo) if p >= 11 else 0))
    return segs


def _plan(segs, L):
    """pieces per segment and the sorted, padded list of (class, length)"""
    keys = []
    for p, kind, cnt in segs:
        if not cnt:
            continue
        path = 0 if p < 2**31 else 1
        T = -(-cnt // L[path])
        n = -(-cnt // T)  # the longest piece
        cls = (2 if p >= 2**31 else (1 if p >= 2**30 else 0)) * 2 + kind
        e = n.bit_length() - 1
        frac = ((n >> (e - 5)) if e >= 5 else (n << (5 - e))) & 31
        keys += [(cls, e * 32 + frac, n)] * T
    keys.sort()
    return keys


def _ids():
    return {wv.wv_congruence_info(c)[0]: c for c in range(wv.wv_congruence_count())}


@pytest.mark.parametrize("lo,hi,names", [
    (1062200000, 1062203000, ("BB2244", "EE2004")),
    (10**11 - 1000, 10**11, ("BB2244", "EE2004")),
    (2**31 - 2000, 2**31 + 2000, ("BB30", "EE33")),
    (5, 3000, ("BB30", "EE33")),
])
def test_piece_count_within_capacity(lo, hi, names):
    ids = _ids()
    cb, ce = ids[names[0]], ids[names[1]]
    primes = oracle.sieve(lo, hi)
    segs = _segments(primes, cb, ce)
    tb, te = wv.wv_count_terms(np.array([p for p in primes if p >= 11], dtype=np.uint64), cb, ce)
    t = [sum(c for p, k, c in segs if p < 2**31), sum(c for p, k, c in segs if p >= 2**31)]
    assert sum(t) == tb + te  # the model counts the library's terms
    target = [SMS * LANES[i] * ROUNDS for i in range(2)]
    L = [max(LMIN[i], -(-t[i] // target[i])) for i in range(2)]
    pieces = _plan(segs, L)
    assert len(pieces) <= len(segs) + sum(target)  # the call's buffer bound
    assert all(n <= L[0 if cls < 4 else 1] for cls, _, n in pieces)
    # a serving plan: L from an O(n) upper bound on the terms, capped
    w = sum((yn / yd - xn / xd) for xn, xd, yn, yd in _rows(cb) + _rows(ce))
    rows = len(_rows(cb)) + len(_rows(ce))
    tub = [sum(w * p + rows for p in primes if p < 2**31), sum(w * p + rows for p in primes if p >= 2**31)]
    assert tub[0] >= t[0] and tub[1] >= t[1]
    Le = []
    for i in range(2):
        want = tub[i] / (ROUNDS_EPOCH * SMS * LANES[i])
        Le.append(max(LMIN[i], LMAX_EPOCH if want > LMAX_EPOCH else int(want) + 1))
    pieces_e = _plan(segs, Le)
    assert len(pieces_e) <= len(segs) + sum(int(tub[i] / Le[i]) + 1 for i in range(2))


def test_sort_keeps_warps_uniform():
    """Pieces sorted by (class, length bin) and each class padded to 32: every
    warp holds one class, and its longest piece is within one bin (2.2 %) of
    its shortest except across bins."""
    ids = _ids()
    primes = np.concatenate([oracle.sieve(10**6, 10**6 + 3000), oracle.sieve(2**30 - 2000, 2**30 + 2000),
                             oracle.sieve(2**31, 2**31 + 1500)])
    segs = _segments(primes, ids["BB249"], ids["EE404"])
    pieces = _plan(segs, [4096, 16384])
    padded, lost, work = [], 0, 0
    for cls in range(6):
        part = [x for x in pieces if x[0] == cls]
        padded += part + [None] * (-len(part) % 32)
    assert len(padded) % 32 == 0
    for w in range(len(padded) // 32):
        lanes = [x for x in padded[32 * w: 32 * w + 32] if x is not None]
        assert lanes and padded[32 * w] is not None        # lane 0 always holds a piece
        assert len({x[0] for x in lanes}) == 1              # one class per warp
        ns = [x[2] for x in lanes]
        work += sum(ns)
        lost += 32 * max(ns) - sum(ns)
    assert work / (work + lost) > 0.9


@pytest.mark.parametrize("n,rows", [(1, 30), (33, 63), (4907, 48), (100, 7), (64, 8)])
def test_chain_kernel_tiles_cover_every_segment_once(n, rows):
    """k_chain_hist / k_chain_scatter: tiles of 8 rows by 32 primes, loaded by
    256 threads prime by prime (thread t: prime t / 8, row t % 8), staged in
    shared memory and read back by warp w, lane l as (row w, prime l).  Every
    segment s = prime * rows + row is loaded exactly once, by eight threads
    reading eight consecutive segments, and each warp reads one row of 32
    consecutive primes."""
    tile_rows, nst = 8, (n + 31) // 32
    nt = ((rows + tile_rows - 1) // tile_rows) * nst
    seen = np.zeros(n * rows, dtype=np.int64)
    for tile in range(nt):
        j0, slot0 = (tile // nst) * tile_rows, (tile % nst) * 32
        stage = {}
        for t in range(256):
            slot, j = slot0 + t // tile_rows, j0 + t % tile_rows
            if slot < n and j < rows:
                seen[slot * rows + j] += 1
                stage[(t % tile_rows, t // tile_rows)] = (slot, j)
        for t in range(0, 256, 8):  # eight threads, one prime, consecutive rows
            segs = [stage[(r, t // 8)] for r in range(8) if (r, t // 8) in stage]
            assert [j for _, j in segs] == list(range(segs[0][1], segs[0][1] + len(segs))) if segs else True
        for w in range(tile_rows):
            for lane in range(32):
                if (w, lane) in stage:
                    assert stage[(w, lane)] == (slot0 + lane, j0 + w)
    assert (seen == 1).all()

