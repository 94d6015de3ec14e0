"""Primality check of caller-supplied prime lists (wv_is_prime, check_primes).

The prime-list entry points take primality as the caller's contract; the
check_primes option makes the planner verify it with a deterministic
Miller-Rabin (bases 2..17, exact below 2^37) and mark composites invalid.
wv_is_prime runs the same test on the host, so it is pinned here against a
sieve, known strong pseudoprimes and Carmichael numbers, without a GPU.
"""
import numpy as np
import pytest

from paper_2101_11157_gb300 import wv


def _sieve(n):
    s = np.ones(n, dtype=bool)
    s[:2] = False
    for q in range(2, int(n ** 0.5) + 1):
        if s[q]:
            s[q * q::q] = False
    return s


def test_is_prime_matches_sieve_below_200000():
    s = _sieve(200_000)
    got = np.array([wv.wv_is_prime(n) for n in range(200_000)])
    assert np.array_equal(got == 1, s)


# composites that pass Miller-Rabin for the first few prime bases (strong
# pseudoprimes: psi_2, psi_3, psi_4, psi_5, psi_6 of Jaeschke's table) and
# Carmichael numbers; all below 2^37
STRONG_PSEUDOPRIMES = [2047, 1373653, 25326001, 3215031751, 2152302898747]
CARMICHAEL = [561, 1105, 1729, 2465, 2821, 6601, 8911, 41041, 825265, 321197185, 5394826801]


def test_pseudoprimes_and_carmichael_numbers_are_composite():
    for n in STRONG_PSEUDOPRIMES + CARMICHAEL:
        want = -1 if n >= 2 ** 37 else 0
        assert wv.wv_is_prime(n) == want, n


def test_range_boundary():
    assert wv.wv_is_prime(2 ** 37) == -1
    assert wv.wv_is_prime(2 ** 64 - 1) == -1
    assert wv.wv_is_prime(2 ** 37 - 1) == 0       # 223 * 616318177
    assert 223 * 616318177 == 2 ** 37 - 1
    assert wv.wv_is_prime(2 ** 37 - 25) == 1       # the largest prime below 2^37
    assert all(wv.wv_is_prime(2 ** 37 - k) == 0 for k in range(1, 25))
    # squares of primes near sqrt(2^37) and products of two such primes
    for a, b in [(370723, 370723), (370723, 370693), (262147, 524269)]:
        assert wv.wv_is_prime(a * b) == 0
    # the Vandiver primes and the Wolstenholme primes below 2^37 (Sec. 1)
    for p in (149, 241, 2946901, 16467631, 17613227, 327784727, 426369739, 1062232319,
              16843, 2124679):
        assert wv.wv_is_prime(p) == 1, p


def test_random_against_sympy():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(20210127)
    ns = rng.integers(2 ** 20, 2 ** 37, size=3000, dtype=np.int64).tolist()
    ns += [n | 1 for n in rng.integers(2 ** 36, 2 ** 37, size=2000, dtype=np.int64).tolist()]
    for n in ns:
        assert wv.wv_is_prime(n) == (1 if sympy.isprime(n) else 0), n


@pytest.mark.gpu
def test_check_primes_marks_composites_invalid():
    import torch
    from paper_2101_11157_gb300 import api
    primes = api.to_u64(api.sieve(1_062_200_000, 1_062_201_000))
    composites = np.array([1_062_200_001, 3215031751, 25326001, 5394826801, 370723 * 370723,
                           2 ** 37 - 1, 321197185], dtype=np.uint64)
    xs = np.concatenate([primes, composites, primes[:3]])
    d = torch.from_numpy(xs.view(np.int64)).cuda()
    ob, oe = torch.empty_like(d), torch.empty_like(d)
    wv.wv_residues_ex(d, ob, oe, {"check_primes": 1})
    torch.cuda.synchronize()
    cb, ce = ob.cpu().numpy().view(np.uint64), oe.cpu().numpy().view(np.uint64)
    pb, pe = torch.empty_like(d), torch.empty_like(d)
    wv.wv_residues_ex(d, pb, pe)
    torch.cuda.synchronize()
    rb, re = pb.cpu().numpy().view(np.uint64), pe.cpu().numpy().view(np.uint64)
    is_p = np.array([wv.wv_is_prime(int(x)) == 1 for x in xs])
    inv = np.uint64(2 ** 64 - 1)
    assert np.array_equal(cb[is_p], rb[is_p]) and np.array_equal(ce[is_p], re[is_p])
    assert np.all(cb[~is_p] == inv) and np.all(ce[~is_p] == inv)
    assert (~is_p).sum() == composites.size
