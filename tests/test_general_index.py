"""General index near the top: B_{p-e} (e odd) and E_{p-1-e} (e even).

CPU: the oracle's general forms (Stafford-Vandiver, eqn 2.4; Glaisher,
eqn 4.1) against the definitions; the library's transcribed general forms
(Vandiver, eqn 2.5; eqn 4.2) evaluated with Python integers against the
definitions.  GPU: wv_residues_general against the oracle, bit for bit, and
against wv_residues_pm3 at e = 3 / 2.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2101_11157_gb300 import wv
from paper_2101_11157_gb300 import workloads as W

SMALL = [p for p in range(11, 420) if W.is_prime(p)]


def test_oracle_general_matches_definitions(orc):
    for p in SMALL[:40]:
        for e in (3, 5, 7, 9, 11):
            if p >= e + 3:
                g = orc.bernoulli_general(p, e)
                assert g == -1 or g == orc.bernoulli_def(p - e, p), (p, e)
        for e in (2, 4, 6, 8, 10):
            if p >= e + 3:
                assert orc.euler_general(p, e) == orc.euler_def(p - 1 - e, p), (p, e)


def test_oracle_general_reduces_to_the_p_minus_3_forms(orc):
    rng = np.random.default_rng(4)
    for x in rng.integers(10**4, 10**6, 6):
        p = W.next_prime(int(x))
        assert orc.bernoulli_general(p, 3) == orc.bernoulli_pm3(p)
        assert orc.euler_general(p, 2) == orc.euler_pm3(p)


def _power_sum(p, x, y, e):
    # sum of s^-e over x p < s < y p, plain Python
    lo = (x.numerator * p) // x.denominator + 1
    hi = -((-y.numerator * p) // y.denominator)  # ceil(y p), exclusive
    return sum(pow(s, -e, p) for s in range(lo, hi)) % p


@pytest.mark.parametrize("kind", [0, 1])
def test_transcribed_general_forms_against_definitions(orc, kind):
    n = wv.wv_general_rows(kind)
    rows = [wv.wv_general_row(kind, r) for r in range(n)]
    assert n == (2 if kind == 0 else 3)
    for p in SMALL[:30]:
        for e in ((3, 5, 7, 9) if kind == 0 else (2, 4, 6, 8)):
            if p < e + 3:
                continue
            rhs = 0
            for (xn, xd, yn, yd), terms, _ in rows:
                coef = sum(c * pow(d, -e, p) for c, d in terms) % p
                rhs += coef * _power_sum(p, Fraction(xn, xd), Fraction(yn, yd), e)
            rhs %= p
            if kind == 0:
                a, b, c = rows[0][2]
                lhs = (pow(a, e, p) + pow(b, e, p) - pow(c, e, p) - 1) * pow(-2 * e, -1, p) % p
                if lhs == 0:
                    continue
                assert rhs == lhs * orc.bernoulli_def(p - e, p) % p, (p, e)
            else:
                lhs = (-1) ** (e // 2) * pow(4, e - 1, p) % p
                assert rhs == lhs * orc.euler_def(p - 1 - e, p) % p, (p, e)


def test_general_rejects_bad_exponents_without_gpu():
    # argument validation happens before any device work
    lib = wv.load()
    for eb, ee in ((4, 0), (1, 0), (17, 0), (0, 3), (0, 18), (0, 1)):
        assert lib.wv_residues_general(None, 0, eb, ee, None, None, None) == wv.WV_EINVAL


@pytest.mark.gpu
def test_gpu_general_small_primes_vs_definitions(orc):
    import torch
    ps = np.array([p for p in range(5, 1200) if W.is_prime(p)], dtype=np.uint64)
    d = torch.from_numpy(ps.view(np.int64)).cuda()
    for eb, ee in ((3, 2), (5, 4), (7, 6), (9, 8), (15, 16)):
        ob, oe = torch.empty_like(d), torch.empty_like(d)
        wv.wv_residues_general(d, eb, ee, ob, oe)
        torch.cuda.synchronize()
        gb, ge = ob.cpu().numpy().view(np.uint64), oe.cpu().numpy().view(np.uint64)
        for i, p in enumerate(ps.tolist()):
            vb = orc.bernoulli_def(p - eb, p) if p >= eb + 3 else None
            ve = orc.euler_def(p - 1 - ee, p) if p >= ee + 3 else None
            lb = (pow(2, eb, p) + pow(5, eb, p) - pow(6, eb, p) - 1) % p
            if p < 11 or vb is None or lb == 0:
                assert gb[i] == wv.WV_RESIDUE_INVALID, (p, eb)
            else:
                assert gb[i] == vb, (p, eb)
            if p < 11 or ve is None:
                assert ge[i] == wv.WV_RESIDUE_INVALID, (p, ee)
            else:
                assert ge[i] == ve, (p, ee)


@pytest.mark.gpu
def test_gpu_general_large_primes_vs_oracle(orc):
    import torch
    rng = np.random.default_rng(12)
    ps = [W.next_prime(int(x)) for x in rng.integers(10**5, 10**7, 10)]
    ps.append(W.next_prime(2**30))  # the 64-bit path
    d = torch.from_numpy(np.array(ps, dtype=np.uint64).view(np.int64)).cuda()
    for eb, ee in ((5, 4), (11, 10)):
        ob, oe = torch.empty_like(d), torch.empty_like(d)
        wv.wv_residues_general(d, eb, ee, ob, oe)
        torch.cuda.synchronize()
        gb, ge = ob.cpu().numpy().view(np.uint64), oe.cpu().numpy().view(np.uint64)
        for i, p in enumerate(ps):
            if p < 2**31:  # the oracle's single sums take ~p/4 modular steps
                assert int(gb[i]) == orc.bernoulli_general(p, eb), (p, eb)
                assert int(ge[i]) == orc.euler_general(p, ee), (p, ee)


@pytest.mark.gpu
def test_gpu_general_at_e3_e2_equals_pm3():
    # two different congruences (Vandiver / eqn 4.2 vs BB30 / EE33) agree on
    # the 4907-prime window near 1.06e9 and on primes beyond 2^30
    import torch
    from paper_2101_11157_gb300 import api
    for lo, hi in (W.P1E9_WINDOW, (2**33, 2**33 + 3000)):
        pr = api.sieve(lo, hi)
        rb, re = api.residues(pr)
        ob, oe = torch.empty_like(pr), torch.empty_like(pr)
        wv.wv_residues_general(pr, 3, 2, ob, oe)
        torch.cuda.synchronize()
        assert torch.equal(ob, rb) and torch.equal(oe, re)
