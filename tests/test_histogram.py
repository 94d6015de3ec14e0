"""Histogram mode (Sec. 3 "Results": 2000 equal bins of <B_{p-3}>_p / p).

CPU: the oracle's binning against a linear scan of the bin edges, its
invariants, and the paper's observation of no bias.  GPU: wv_histogram against
the oracle's binning of the oracle's residues, bit-exact counts.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2101_11157_gb300 import workloads as W


def _scan_bin(p, r, bins, orc):
    u = Fraction(orc.symmetric(r, p), p) + Fraction(1, 2)
    for b in range(bins):
        if Fraction(b, bins) <= u < Fraction(b + 1, bins):
            return b
    raise AssertionError("u outside [0, 1)")


def test_oracle_histogram_matches_edge_scan(orc):
    rng = np.random.default_rng(3)
    for bins in (1, 2, 7, 2000):
        ps = [5, 7, 11, 13, 149, 16843] + [W.next_prime(int(x)) for x in rng.integers(20, 10**9, 40)]
        rs = [0, 1, 2, 3] + [int(rng.integers(0, p)) for p in ps[4:]]
        rs += [0] * (len(ps) - len(rs))
        h = orc.histogram(ps, rs, bins)
        want = np.zeros(bins, dtype=np.int64)
        for p, r in zip(ps, rs):
            want[_scan_bin(p, r, bins, orc)] += 1
        assert np.array_equal(h, want)
        assert h.sum() == len(ps)


def test_oracle_histogram_symmetry_and_zero(orc):
    # <r> and <-r> fall in mirrored bins; r = 0 (a Wolstenholme / Vandiver
    # prime) sits at u = 1/2, the lower edge of bin bins/2
    p, bins = 1_000_003, 2000
    for r in (1, 17, 499_999, 500_001, 123_456):
        a = np.flatnonzero(orc.histogram([p], [r], bins))[0]
        b = np.flatnonzero(orc.histogram([p], [p - r], bins))[0]
        assert a + b == bins - 1
    assert np.flatnonzero(orc.histogram([16843], [0], bins))[0] == bins // 2


def test_oracle_histogram_no_bias_small_primes(orc):
    # the paper sees no bias in B_{p-3} mod p; with 5131 primes below 5e4 and
    # 20 bins every count lies within 5 standard deviations of 5131/20
    ps = orc.sieve(5, 50_000)
    rb, re = orc.residues(ps)
    for res in (rb, re):
        h = orc.histogram(ps, res, 20)
        mean, sd = len(ps) / 20, (len(ps) / 20 * (1 - 1 / 20)) ** 0.5
        assert h.sum() == len(ps)
        assert np.all(np.abs(h - mean) < 5 * sd), h


@pytest.mark.gpu
def test_gpu_histogram_matches_oracle(orc):
    import torch
    from paper_2101_11157_gb300 import wv
    ps = orc.sieve(5, 50_000)
    rb, re = orc.residues(ps)
    for bins in (2000, 1, 7, 10_000):
        hb = torch.zeros(bins, dtype=torch.int64, device="cuda")
        he = torch.zeros_like(hb)
        n = wv.wv_histogram(5, 50_000, hb, he)
        assert n == len(ps)
        assert np.array_equal(hb.cpu().numpy(), orc.histogram(ps, rb, bins))
        assert np.array_equal(he.cpu().numpy(), orc.histogram(ps, re, bins))
    # accumulation over disjoint ranges equals one call; one kind only
    hb = torch.zeros(2000, dtype=torch.int64, device="cuda")
    wv.wv_histogram(5, 20_000, hb, None)
    wv.wv_histogram(20_000, 50_000, hb, None)
    assert np.array_equal(hb.cpu().numpy(), orc.histogram(ps, rb, 2000))


@pytest.mark.gpu
def test_gpu_histogram_p1e9_window(orc):
    # the bench window: binning of the GPU's own residues (parity of the
    # residues themselves is checked elsewhere) and of the known Vandiver prime
    import torch
    from paper_2101_11157_gb300 import api, wv
    lo, hi = W.P1E9_WINDOW
    _, pr, rb, re = api.search(lo, hi, with_residues=True)
    hb = torch.zeros(2000, dtype=torch.int64, device="cuda")
    he = torch.zeros_like(hb)
    assert wv.wv_histogram(lo, hi, hb, he) == pr.numel()
    ps = api.to_u64(pr)
    assert np.array_equal(hb.cpu().numpy(), orc.histogram(ps, api.to_u64(rb), 2000))
    assert np.array_equal(he.cpu().numpy(), orc.histogram(ps, api.to_u64(re), 2000))
    assert he[1000].item() >= 1  # E residue 0 at 1062232319 -> u = 1/2


@pytest.mark.gpu
def test_gpu_histogram_rejects_bad_bins():
    import torch
    from paper_2101_11157_gb300 import wv
    with pytest.raises(wv.WvError):
        wv.wv_histogram(5, 100, None, None)
