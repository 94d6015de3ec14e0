"""Pins for the oracle's plain sieve: Miller-Rabin (a different algorithm) on
windows, and the textbook count pi(50000) = 5133."""
import numpy as np
import pytest

from paper_2101_11157_gb300 import workloads as W


@pytest.mark.parametrize("lo,hi", [(0, 5000), (5, 50_000), (10**9, 10**9 + 3000),
                                   (2**31 - 2000, 2**31 + 2000), (10**11 - 3000, 10**11)])
def test_sieve_matches_miller_rabin(orc, lo, hi):
    got = orc.sieve(lo, hi)
    ref = W.primes_in(lo, hi)
    assert np.array_equal(got, ref)


def test_sieve_textbook_count(orc):
    assert orc.sieve(0, 50_000).size == 5133          # pi(5e4)
    assert orc.sieve(5, 50_000).size == 5131


def test_sieve_edges(orc):
    assert orc.sieve(10, 10).size == 0
    assert orc.sieve(24, 29).size == 0
    assert list(orc.sieve(0, 12)) == [2, 3, 5, 7, 11]
    assert list(orc.sieve(2, 3)) == [2]
