"""The serving loop: queries submitted while others run share epochs on the
device (continuous batching); each result equals the same query computed
alone, bit for bit, and the CPU oracle's residues (computed here for small
primes, stored by tests/golden/make_oracle_residues.py for large ones)."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from conftest import read_golden  # noqa: E402
from paper_2101_11157_gb300 import api, wv  # noqa: E402

TOP_PRIME = 99_999_998_237  # one of the 8 stored primes of [1e11 - 1e4, 1e11)


def _gold():
    out = {}
    for name in ("serve_sample_residues.txt", "top_window_subset_residues.txt"):
        out.update({int(p): (int(b), int(e)) for p, b, e in read_golden(name)})
    return out


def _oracle_check(orc, gold, pr, rb, re):
    """Compare a served result with the oracle: every prime below 1e8 of a
    small result (a seeded sample of 24 of a larger one) recomputed here, and
    every prime with stored residues.  Returns how many primes were checked."""
    small = [i for i, p in enumerate(pr) if int(p) < 10**8]
    if len(small) > 24:
        small = sorted(np.random.default_rng(3).choice(small, 24, replace=False))
    n = 0
    if small:
        ob, oe = orc.residues(pr[small])
        assert np.array_equal(rb[small], ob) and np.array_equal(re[small], oe)
        n += len(small)
    for i, p in enumerate(pr):
        if int(p) in gold:
            assert (int(rb[i]), int(re[i])) == gold[int(p)], int(p)
            n += 1
    return n


def _alone_range(lo, hi):
    lo = max(lo, 5)
    if hi <= lo:
        return (np.zeros(0, np.uint64),) * 3
    _, pr, rb, re = api.search(lo, hi, with_residues=True)
    torch.cuda.synchronize()
    return api.to_u64(pr), api.to_u64(rb), api.to_u64(re)


def _alone_prime(p):
    d = torch.tensor([p], dtype=torch.int64, device="cuda")
    rb, re = api.residues(d)
    torch.cuda.synchronize()
    return np.array([p], np.uint64), api.to_u64(rb), api.to_u64(re)


QUERIES = [("range", 2 * 10**9, 2 * 10**9 + 600000),  # long-running (~1 s), 64-bit path
           ("prime", 1062232319, None),                  # the Vandiver prime
           ("range", 5, 3000),
           ("prime", 16843, None),                       # the Wolstenholme prime
           ("range", 10**7, 10**7 + 20000),
           ("prime", 2**30 + 3, None),
           ("range", 999_999_000, 1_000_001_000),
           ("prime", TOP_PRIME, None),                   # near the top of the search range
           ("range", 10, 10)]                            # empty


def _run(server, stagger):
    ids = []
    for i, (kind, a, b) in enumerate(QUERIES):
        ids.append(wv.wv_server_submit_range(server, a, b) if kind == "range"
                   else wv.wv_server_submit_prime(server, a))
        if stagger and i == 0:
            time.sleep(0.05)  # the first query is already on the device when the rest arrive
    infos = [wv.wv_server_wait(server, q, 300.0) for q in ids]
    return ids, infos


def test_serving_results_equal_alone_and_overlap(orc):
    gold = _gold()
    s = wv.wv_server_create(epoch_terms=2e9)
    try:
        ids, infos = _run(s, stagger=True)
        for (kind, a, b), q, info in zip(QUERIES, ids, infos):
            assert info["state"] == 2
            pr, rb, re = wv.wv_server_result(s, q)
            ref = _alone_range(a, b) if kind == "range" else _alone_prime(a)
            assert np.array_equal(pr, ref[0]) and np.array_equal(rb, ref[1]) and np.array_equal(re, ref[2])
            assert info["n_primes"] == pr.size
            # against the oracle: every non-empty query has primes it checks
            assert _oracle_check(orc, gold, pr, rb, re) >= min(pr.size, 1), (kind, a, b)
        # the long range's primes are the oracle's sieve of it
        assert orc.sieve(2 * 10**9, 2 * 10**9 + 600000).tolist() == wv.wv_server_result(s, ids[0])[0].tolist()
        # the known zeros came back
        assert wv.wv_server_result(s, ids[1])[2][0] == 0
        assert wv.wv_server_result(s, ids[3])[1][0] == 0
        st = wv.wv_server_stats(s)
        assert st["peak_active"] >= 2 and st["epochs"] >= 2 and st["bytes_in_use"] == 0
        # the small queries submitted behind the long one finished before it
        assert infos[2]["t_done"] < infos[0]["t_done"]
    finally:
        wv.wv_server_destroy(s)


def test_serving_under_a_tight_memory_budget():
    s = wv.wv_server_create(mem_budget=8 << 20, max_active=3, epoch_terms=1e9)
    try:
        ids, infos = _run(s, stagger=False)
        for (kind, a, b), q, info in zip(QUERIES, ids, infos):
            pr, rb, re = wv.wv_server_result(s, q)
            ref = _alone_range(a, b) if kind == "range" else _alone_prime(a)
            assert np.array_equal(rb, ref[1]) and np.array_equal(re, ref[2])
        assert wv.wv_server_stats(s)["bytes_in_use"] == 0
    finally:
        wv.wv_server_destroy(s)


def test_small_query_backfills_past_a_blocked_large_one():
    # the budget holds one of the two large ranges at a time; the single prime
    # submitted behind the second one is admitted (and done) before it
    s = wv.wv_server_create(mem_budget=20 << 20, epoch_terms=2e10)
    try:
        a = wv.wv_server_submit_range(s, 2 * 10**9, 2 * 10**9 + 30000)
        time.sleep(0.05)
        b = wv.wv_server_submit_range(s, 2 * 10**9 + 30000, 2 * 10**9 + 60000)
        c = wv.wv_server_submit_prime(s, 1062232319)
        ia, ib, ic = (wv.wv_server_wait(s, q, 300.0) for q in (a, b, c))
        assert ic["t_admit"] < ib["t_admit"] and ic["t_done"] < ib["t_admit"]
        assert ib["t_admit"] >= ia["t_done"] - 1e-3
        gold = _gold()
        for q, (lo, hi) in ((a, (2 * 10**9, 2 * 10**9 + 30000)), (b, (2 * 10**9 + 30000, 2 * 10**9 + 60000))):
            pr, rb, re = wv.wv_server_result(s, q)
            ref = _alone_range(lo, hi)
            assert np.array_equal(pr, ref[0]) and np.array_equal(rb, ref[1]) and np.array_equal(re, ref[2])
            assert sum(int(p) in gold for p in pr) == 6
            assert _oracle_check(None, gold, pr, rb, re) == 6
        assert wv.wv_server_result(s, c)[2][0] == 0
    finally:
        wv.wv_server_destroy(s)


def test_serving_rejects_bad_queries():
    s = wv.wv_server_create()
    try:
        with pytest.raises(wv.WvError):
            wv.wv_server_submit_prime(s, 4)
        with pytest.raises(wv.WvError):
            wv.wv_server_submit_range(s, 10, 2**38)
    finally:
        wv.wv_server_destroy(s)


def test_serving_rejects_bad_configs():
    for kw in ({"epoch_form": 4}, {"epoch_block": 48}, {"epoch_block": 512}, {"piece_log2": 11},
               {"piece_log2": 25}):
        with pytest.raises(wv.WvError):
            wv.wv_server_destroy(wv.wv_server_create(**kw))


@pytest.mark.parametrize("k", [12, 20])
def test_serving_piece_length_keeps_results(k):
    """Pieces of at most 2^12 (many per sum, short u-form pieces) and 2^20
    terms (whole sums): the same residues as the query computed alone, and the
    stored oracle residues of a prime below 1e11."""
    s = wv.wv_server_create(piece_log2=k, epoch_terms=2e10)
    try:
        a = wv.wv_server_submit_range(s, 2 * 10**9, 2 * 10**9 + 20000)
        b = wv.wv_server_submit_prime(s, TOP_PRIME)
        for q in (a, b):
            assert wv.wv_server_wait(s, q, 600.0)["state"] == 2
        pr, rb, re = wv.wv_server_result(s, a)
        ref = _alone_range(2 * 10**9, 2 * 10**9 + 20000)
        assert np.array_equal(pr, ref[0]) and np.array_equal(rb, ref[1]) and np.array_equal(re, ref[2])
        pr, rb, re = wv.wv_server_result(s, b)
        assert (int(rb[0]), int(re[0])) == _gold()[TOP_PRIME]
    finally:
        wv.wv_server_destroy(s)
