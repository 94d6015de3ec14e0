"""The calls the benchmark times, against residues the CPU oracle stored.

tests/golden/make_oracle_residues.py wrote, with the oracle alone (B_{p-3} by
the Stafford-Vandiver congruence, eqn 2.4; E_{p-3} by Glaisher's congruence,
eqn 4.1), the residues of every prime of the 1e5-wide window at 1.06e9 and of
the 8 seeded primes of [1e11 - 1e4, 1e11).  Here the CUDA path, through the C
ABI, must give exactly those values: the search as the benchmark runs it (the
congruences it picks by range: BB2244 + EE2004 at 1.06e9, BB3802 + EE4122
near 1e11), the default of a device prime list (BB30 + EE33), and each
hot-loop formulation of both arithmetic paths."""
import numpy as np
import pytest

from conftest import read_golden
from paper_2101_11157_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11157_gb300 import api, wv  # noqa: E402


def _gold(name):
    rows = read_golden(name)
    p = np.array([int(r[0]) for r in rows], dtype=np.uint64)
    b = np.array([int(r[1]) for r in rows], dtype=np.uint64)
    e = np.array([int(r[2]) for r in rows], dtype=np.uint64)
    return p, b, e


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _residues(primes, options=None):
    d = _dev(primes)
    rb, re = api.residues(d, options=options)
    torch.cuda.synchronize()
    return api.to_u64(rb), api.to_u64(re)


def _bench_step(lo, hi):
    """wv_search_ex over [lo, hi) with the residue buffers, as bench.py times it."""
    n = wv.wv_sieve_count(lo, hi)
    hits = torch.empty((64, 2), dtype=torch.int64, device="cuda")
    d_pr = torch.empty(n, dtype=torch.int64, device="cuda")
    d_rb, d_re = torch.empty_like(d_pr), torch.empty_like(d_pr)
    nh, npr = wv.wv_search_ex(lo, hi, 0, hits, d_pr, d_rb, d_re, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert npr == n
    return nh, api.to_u64(d_pr), api.to_u64(d_rb), api.to_u64(d_re)


def test_p1e9_window_bench_step_equals_oracle():
    gp, gb, ge = _gold("p1e9_window_residues.txt")
    assert gp.size == 4907
    cb, ce = wv.wv_congruence_for_range(*W.P1E9_WINDOW)
    assert [wv.wv_congruence_info(c)[0] for c in (cb, ce)] == ["BB2244", "EE2004"]
    nh, pr, rb, re = _bench_step(*W.P1E9_WINDOW)
    assert np.array_equal(pr, gp)
    assert np.array_equal(rb, gb)
    assert np.array_equal(re, ge)
    assert nh == 1 and int(ge[np.searchsorted(gp, W.KNOWN_VANDIVER_IN_P1E9)]) == 0


@pytest.mark.parametrize("opt", [None, {"arith": 9}, {"arith": 29}, {"arith": 30},
                                 {"arith": 31, "ilp": 1}, {"arith": 4}])
def test_p1e9_window_formulations_equal_oracle(opt):
    """The window's congruences under the default and the other 32-bit
    formulations, and the device-list default BB30 + EE33."""
    gp, gb, ge = _gold("p1e9_window_residues.txt")
    cb, ce = wv.wv_congruence_for_range(*W.P1E9_WINDOW)
    rb, re = _residues(gp, {**(opt or {}), "cong_b": cb, "cong_e": ce})
    assert np.array_equal(rb, gb) and np.array_equal(re, ge)
    rb, re = _residues(gp, opt)
    assert np.array_equal(rb, gb) and np.array_equal(re, ge)


def test_top_window_bench_step_equals_oracle():
    gp, gb, ge = _gold("top_window_subset_residues.txt")
    assert gp.size == 8 and np.array_equal(gp, W.top_window_subset(seed=5, k=8))
    cb, ce = wv.wv_congruence_for_range(*W.TOP_WINDOW)
    assert [wv.wv_congruence_info(c)[0] for c in (cb, ce)] == ["BB3802", "EE4122"]
    nh, pr, rb, re = _bench_step(*W.TOP_WINDOW)
    assert pr.size == 391 and nh == 0  # no Wolstenholme or Vandiver prime there (Theorem 1.1)
    idx = np.searchsorted(pr, gp)
    assert np.array_equal(pr[idx], gp)
    assert np.array_equal(rb[idx], gb)
    assert np.array_equal(re[idx], ge)


@pytest.mark.parametrize("opt", [None, {"arith": 1}, {"arith": 21}, {"arith": 32}, {"arith": 33},
                                 {"arith": 37}, {"arith": 38}, {"arith": 49}, {"arith": 50}])
def test_top_window_formulations_equal_oracle(opt):
    """The 8 stored primes below 1e11 on the 64-bit path: the device-list
    default (BB30 + EE33) and the range's congruences, under the default, the
    single-term form and other grouped 64-bit formulations."""
    gp, gb, ge = _gold("top_window_subset_residues.txt")
    rb, re = _residues(gp, opt)
    assert np.array_equal(rb, gb) and np.array_equal(re, ge)
    if opt is None or opt.get("arith") != 1:  # the single-term form is slow on the long sums
        cb, ce = wv.wv_congruence_for_range(*W.TOP_WINDOW)
        rb, re = _residues(gp, {**(opt or {}), "cong_b": cb, "cong_e": ce})
        assert np.array_equal(rb, gb) and np.array_equal(re, ge)


@pytest.mark.parametrize("opt", [None, {"arith": 40}, {"arith": 39}, {"arith": 31, "ilp": 2},
                                 {"arith": 44}, {"arith": 45}, {"arith": 46}, {"arith": 47},
                                 {"arith": 45, "ilp": 2}, {"arith": 48}, {"tiling": 1},
                                 {"tiling": 1, "arith": 31, "ilp": 2}])
def test_p1e9_window_work_units_equal_oracle(opt):
    """The window under lane chains (the default: each lane sums its own piece
    of a sum, pieces sorted by length) with the lane formulations, and under
    warp tiles, against the stored oracle residues."""
    gp, gb, ge = _gold("p1e9_window_residues.txt")
    cb, ce = wv.wv_congruence_for_range(*W.P1E9_WINDOW)
    rb, re = _residues(gp, {**(opt or {}), "cong_b": cb, "cong_e": ce})
    assert np.array_equal(rb, gb) and np.array_equal(re, ge)


@pytest.mark.parametrize("opt", [None, {"arith": 42}, {"arith": 43}, {"arith": 49}, {"arith": 50},
                                 {"tiling": 1}])
def test_lane_chains_few_primes_equal_oracle(opt):
    """Lists of 1 to 8 stored primes below 1e11 and the first 33 of the window at
    1.06e9: most lanes of the last warp of a class are padding, the sums split
    into many pieces (few primes, many lanes), and the paths mix."""
    tp, tb, te = _gold("top_window_subset_residues.txt")
    wp, wb, we = _gold("p1e9_window_residues.txt")
    cb, ce = wv.wv_congruence_for_range(*W.TOP_WINDOW)
    for k in (1, 2, 5, 8):
        rb, re = _residues(tp[:k], {**(opt or {}), "cong_b": cb, "cong_e": ce})
        assert np.array_equal(rb, tb[:k]) and np.array_equal(re, te[:k]), k
    for k in (1, 31, 32, 33):
        rb, re = _residues(wp[:k], {**(opt or {}), "cong_b": cb, "cong_e": ce})
        assert np.array_equal(rb, wb[:k]) and np.array_equal(re, we[:k]), k
    mix = np.concatenate([wp[:33], tp[:3]])
    rb, re = _residues(mix, opt)
    assert np.array_equal(rb, np.concatenate([wb[:33], tb[:3]]))
    assert np.array_equal(re, np.concatenate([we[:33], te[:3]]))
