"""Pins for the CPU oracle, each against something other than the oracle itself:
library routines (sympy), floating-point evaluation of the generating
functions, textbook values, closed-form congruences, the paper's printed
values and brute force.  A plausible slip in any level (a dropped term, a
sign, an index, the sec/sech convention) fails at least one test here."""
import math
from fractions import Fraction

import pytest

from conftest import read_golden
from paper_2101_11157_gb300.workloads import is_prime

SMALL_PRIMES = [p for p in range(5, 1200) if is_prime(p)]


# --------------------------------------------------------------------------
# exact rationals (Sec. 1 generating functions)
# --------------------------------------------------------------------------
def test_exact_textbook_values(orc):
    assert orc.exact_bernoulli(0) == 1
    assert orc.exact_bernoulli(1) == Fraction(-1, 2)   # z/(e^z-1) convention
    assert orc.exact_bernoulli(2) == Fraction(1, 6)
    assert orc.exact_bernoulli(4) == Fraction(-1, 30)
    assert orc.exact_bernoulli(12) == Fraction(-691, 2730)
    assert orc.exact_bernoulli(3) == 0 and orc.exact_bernoulli(25) == 0
    # sec convention: all even-index values positive
    assert [orc.exact_euler(n) for n in range(0, 12, 2)] == [1, 1, 5, 61, 1385, 50521]
    assert orc.exact_euler(7) == 0


def test_exact_against_generating_functions_numerically(orc):
    # z/(e^z - 1) and sec z evaluated in floating point at a few points
    for z in (0.3, 0.7, 1.1):
        b = sum(float(orc.exact_bernoulli(k)) * z ** k / math.factorial(k) for k in range(60))
        assert abs(b - z / math.expm1(z)) < 1e-12
        e = sum(orc.exact_euler(k) * z ** k / math.factorial(k) for k in range(120))
        assert abs(e - 1.0 / math.cos(z)) < 1e-9


def test_exact_against_sympy(orc):
    sympy = pytest.importorskip("sympy")
    for n in range(0, 61, 2):
        assert orc.exact_bernoulli(n) == Fraction(int(sympy.bernoulli(n).p), int(sympy.bernoulli(n).q))
        # sympy uses the sech convention: E_n(sec) = (-1)^(n/2) E_n(sech)
        assert orc.exact_euler(n) == (-1) ** (n // 2) * int(sympy.euler(n))


# --------------------------------------------------------------------------
# Level A: the recurrences reduced mod p, against the exact values
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", [p for p in SMALL_PRIMES if p < 260])
def test_level_a_matches_exact(orc, p):
    assert orc.bernoulli_def(p - 3, p) == orc.rational_mod(orc.exact_bernoulli(p - 3), p)
    assert orc.euler_def(p - 3, p) == orc.exact_euler(p - 3) % p
    # other indices too, so an off-by-one in the target index cannot hide
    for n in (2, 4, 10, p - 5):
        if 0 < n < p - 1:
            assert orc.bernoulli_def(n, p) == orc.rational_mod(orc.exact_bernoulli(n), p)
            assert orc.euler_def(n, p) == orc.exact_euler(n) % p


# --------------------------------------------------------------------------
# Level B: Glaisher (eqn 1.2) and the harmonic sum (eqn 1.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", SMALL_PRIMES[:140])
def test_level_b_matches_definition(orc, p):
    ref = orc.bernoulli_def(p - 3, p)
    assert orc.bernoulli_glaisher(p, 2) == ref
    assert orc.bernoulli_glaisher(p, 3) == ref
    if p != 5:
        assert orc.bernoulli_glaisher(p, 5) == ref
    assert orc.bernoulli_h2(p) == ref


def test_wolstenholme_definition_eqn_1_1(orc):
    # all three congruences of eqn 1.1 hold at 16843 and at no other prime near it
    assert orc.wolstenholme_bits(16843) == 7
    for p in [p for p in range(16000, 17500) if is_prime(p) and p != 16843]:
        assert orc.wolstenholme_bits(p) == 0
    for p in SMALL_PRIMES[:60]:
        assert orc.wolstenholme_bits(p) == 0


# --------------------------------------------------------------------------
# Level C: single-sum congruences (eqns 2.4, 2.8, 4.1, 4.7) vs the definition
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", SMALL_PRIMES)
def test_level_c_matches_definition(orc, p):
    rb = orc.bernoulli_def(p - 3, p)
    re_ = orc.euler_def(p - 3, p)
    if p != 7:
        assert orc.bernoulli_sv(p) == rb
    if p >= 7:
        assert orc.bernoulli_v12(p) == rb
        assert orc.euler_mcintosh(p) == re_
    assert orc.euler_glaisher(p) == re_
    assert orc.bernoulli_pm3(p) == rb
    assert orc.euler_pm3(p) == re_


def test_eqn_4_1_printed_sign_fails_for_p_3_mod_4(orc):
    """The printed factor (-1)^{(p-1)/2-k} at k=1 disagrees with the definition
    exactly when p = 3 mod 4; the factor (-1)^k agrees for every p."""
    for p in SMALL_PRIMES[:80]:
        S = orc.interval_sum(p, Fraction(0), Fraction(1, 4), 2)
        ref = orc.euler_def(p - 3, p)
        printed = S * pow((-1) ** ((p - 1) // 2 - 1) * 4, -1, p) % p
        read = S * pow(-4, -1, p) % p
        assert read == ref
        if ref != 0:
            assert (printed == ref) == (p % 4 == 1)


def test_level_c_cross_forms_mid_range(orc):
    # independent forms agree at primes far beyond the O(p^2) definition
    for p in (100_003, 250_007, 1_000_003, 3_000_017):
        assert is_prime(p)
        b = orc.bernoulli_sv(p)
        assert orc.bernoulli_v12(p) == b
        assert orc.bernoulli_h2(p) == b
        assert orc.euler_mcintosh(p) == orc.euler_glaisher(p)


# --------------------------------------------------------------------------
# the paper's printed values (Theorem 1.1, Tables 1-2)
# --------------------------------------------------------------------------
def _known():
    rows = read_golden("known_primes.txt")
    return [(k, int(p)) for k, p in rows]


def test_known_wolstenholme_and_vandiver_primes(orc):
    for kind, p in _known():
        if p > 2e7:
            continue  # the larger ones are covered by the threaded test below
        if kind == "W":
            assert orc.bernoulli_pm3(p) == 0
            assert orc.bernoulli_v12(p) == 0
        elif kind == "V":
            assert orc.euler_pm3(p) == 0
            assert orc.euler_mcintosh(p) == 0
        elif kind == "notV":
            assert orc.euler_pm3(p) != 0


def test_small_scan_hits(orc):
    """Every prime 5 <= p < 30000: zero residues exactly at the known primes."""
    from paper_2101_11157_gb300.workloads import primes_in
    ps = primes_in(5, 30000)
    b, e = orc.residues(ps)
    assert [int(p) for p, r in zip(ps, b) if r == 0] == [16843]
    assert [int(p) for p, r in zip(ps, e) if r == 0] == [149, 241]


def test_near_miss_and_large_known_primes(orc):
    """Threaded: two rows of Table 1, and the Vandiver primes 3.2e8 and 4.3e8."""
    rows_b = [(int(p), int(v)) for p, v in read_golden("near_miss_bernoulli.txt")][:2]
    big_v = [p for k, p in _known() if k == "V" and 2e7 < p < 5e8]
    ps = [p for p, _ in rows_b]
    b, _ = orc.residues(ps, method_b="default", method_e=None, threads=len(ps))
    for (p, v), r in zip(rows_b, b):
        assert orc.symmetric(int(r), p) == v
    _, e = orc.residues(big_v, method_b=None, method_e="default", threads=len(big_v))
    assert [int(x) for x in e] == [0] * len(big_v)
