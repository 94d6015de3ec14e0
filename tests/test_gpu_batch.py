"""Batched residues (one graph-captured launch sequence over many requests)
against one wv_residues_pm3 call per request, bit for bit."""
import numpy as np
import pytest

from paper_2101_11157_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11157_gb300 import api, wv  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _single(d):
    rb, re = torch.empty_like(d), torch.empty_like(d)
    wv.wv_residues_pm3(d, rb, re)
    return rb, re


def test_batch_matches_single_requests_and_replays():
    # uneven requests: tiny primes, mid-size, both sides of 2^30, one 1-prime request
    lists = [np.array([5, 7, 11, 13, 149], dtype=np.uint64),
             api.to_u64(api.sieve(10**6, 10**6 + 2000)),
             api.to_u64(api.sieve(2**30 - 3000, 2**30 + 3000)),
             np.array([1062232319], dtype=np.uint64),
             api.to_u64(api.sieve(3 * 10**9, 3 * 10**9 + 500))]
    reqs = []
    for a in lists:
        d = _dev(a)
        reqs.append((d, torch.full_like(d, -1), torch.full_like(d, -1)))
    b = wv.wv_batch_create(reqs)
    nreq, nprimes, nodes = wv.wv_batch_info(b)
    assert nreq == len(lists) and nprimes == sum(a.size for a in lists) and nodes > 5
    for rep in range(2):
        for d, ob, oe in reqs:
            ob.fill_(-1)
            oe.fill_(-1)
        wv.wv_batch_run(b)
        torch.cuda.synchronize()
        for d, ob, oe in reqs:
            rb, re = _single(d)
            torch.cuda.synchronize()
            assert torch.equal(ob, rb) and torch.equal(oe, re)
    # new data in the same buffers is picked up by a replay
    d0 = reqs[1][0]
    d0.copy_(_dev(api.to_u64(api.sieve(5 * 10**6, 5 * 10**6 + 40000))[:d0.numel()]))
    wv.wv_batch_run(b)
    torch.cuda.synchronize()
    rb, re = _single(d0)
    assert torch.equal(reqs[1][1], rb) and torch.equal(reqs[1][2], re)
    wv.wv_batch_destroy(b)


def test_batch_seeded_requests():
    reqs_np = W.batch_requests(seed=7, k=16, hi=2e8, max_len=64)
    reqs = [(_dev(a),) for a in reqs_np]
    reqs = [(d, torch.empty_like(d), torch.empty_like(d)) for (d,) in reqs]
    b = wv.wv_batch_create(reqs, {"tile_terms": 4096, "max_tiles": 64})
    wv.wv_batch_run(b)
    torch.cuda.synchronize()
    for d, ob, oe in reqs:
        rb, re = _single(d)
        torch.cuda.synchronize()
        assert torch.equal(ob, rb) and torch.equal(oe, re)
    wv.wv_batch_destroy(b)


def test_autotuner_picks_a_shape_with_identical_results():
    from paper_2101_11157_gb300 import tune
    reqs_np = W.batch_requests(seed=7, k=6, max_len=64)
    reqs = []
    for a in reqs_np:
        d = torch.from_numpy(a.view(np.int64)).cuda()
        reqs.append((d, torch.empty_like(d), torch.empty_like(d)))
    best, table = tune.tune_batch(reqs, grid=[{}, {"block": 32}, {"ilp": 1}], reps=1)
    assert len(table) == 3 and all(r["identical"] for r in table)
    assert best in [r["options"] for r in table]
    b = wv.wv_batch_create(reqs, best or None)
    try:
        wv.wv_batch_run(b)
        torch.cuda.synchronize()
    finally:
        wv.wv_batch_destroy(b)
    for (d, rb, re), a in zip(reqs, reqs_np):
        gb, ge = api.residues(d)
        assert torch.equal(rb, gb) and torch.equal(re, ge)


def _golden_map(name):
    from conftest import read_golden
    return {int(p): (int(b), int(e)) for p, b, e in read_golden(name)}


def test_full_seed7_batch_against_oracle():
    """The whole seed-7 workload (64 requests of 1..4096 primes drawn
    log-uniformly from [1e5, 1e10)) in one batch: a sample of two primes per
    request against residues stored by the oracle (B by eqn 2.4, E by eqn 4.1),
    and every request against the per-request call."""
    reqs_np = W.batch_requests(seed=7)
    assert len(reqs_np) == 64 and max(a.size for a in reqs_np) <= 4096
    gold = _golden_map("batch_seed7_sample_residues.txt")
    reqs = []
    for a in reqs_np:
        d = _dev(a)
        reqs.append((d, torch.full_like(d, -1), torch.full_like(d, -1)))
    b = wv.wv_batch_create(reqs)
    try:
        wv.wv_batch_run(b)
        torch.cuda.synchronize()
    finally:
        wv.wv_batch_destroy(b)
    checked = set()
    for a, (d, ob, oe) in zip(reqs_np, reqs):
        gb, ge = api.to_u64(ob), api.to_u64(oe)
        hit = [i for i, p in enumerate(a) if int(p) in gold]
        assert hit, "every request has a stored oracle sample"
        for i in hit:
            assert (int(gb[i]), int(ge[i])) == gold[int(a[i])], int(a[i])
            checked.add(int(a[i]))
        rb, re = _single(d)
        torch.cuda.synchronize()
        assert torch.equal(ob, rb) and torch.equal(oe, re)
    assert checked == set(gold) and len(checked) >= 64
