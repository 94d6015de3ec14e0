"""Seeded synthetic workloads for the Wolstenholme/Vandiver residue search.

This module holds input generators only: prime windows, seeded prime lists,
batched request sets and serving streams.  It contains none of the residue
arithmetic, and both the CUDA path's tests/benchmarks and the CPU oracle's
tests draw their inputs from it.  Primality here is a deterministic
Miller-Rabin test used only to *generate* inputs.

The paper uses no dataset: its search runs over every prime below 1e11
(Sec. 3 "Results", Sec. 5).  The workloads below are windows and seeded
samples of that same prime range.
"""
from __future__ import annotations

import math

import numpy as np

# Windows of the search range (half-open [lo, hi)).
SMALL_WINDOW = (5, 50_000)                       # all primes 5 <= p < 5e4
P1E9_WINDOW = (1_062_200_000, 1_062_300_000)     # 1e5-wide window near 1.06e9
TOP_WINDOW = (10**11 - 10**4, 10**11)            # top of the paper's search bound

KNOWN_VANDIVER_IN_P1E9 = 1_062_232_319

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)  # deterministic below 3.3e24
_SMALL = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24."""
    if n < 2:
        return False
    for q in _SMALL:
        if n % q == 0:
            return n == q
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def next_prime(n: int) -> int:
    """Smallest prime >= n."""
    n = max(int(n), 2)
    while not is_prime(n):
        n += 1
    return n


def primes_in(lo: int, hi: int) -> np.ndarray:
    """All primes in [lo, hi) by Miller-Rabin (for windows of modest width)."""
    return np.array([v for v in range(max(lo, 2), hi) if is_prime(v)], dtype=np.uint64)


def seeded_subset(primes, k: int, seed: int, must_include=()) -> np.ndarray:
    """k primes drawn without replacement (numpy default_rng(seed)), plus any
    `must_include` values, sorted ascending."""
    primes = np.asarray(primes, dtype=np.uint64)
    rng = np.random.default_rng(seed)
    k = min(k, primes.size)
    idx = rng.choice(primes.size, size=k, replace=False)
    out = set(int(v) for v in primes[idx]) | set(int(v) for v in must_include)
    return np.array(sorted(out), dtype=np.uint64)


def top_window_subset(seed: int = 5, k: int = 8) -> np.ndarray:
    """Seeded subset of the primes in [1e11 - 1e4, 1e11)."""
    return seeded_subset(primes_in(*TOP_WINDOW), k, seed)


def batch_requests(seed: int = 7, k: int = 64, lo: float = 1e5, hi: float = 1e10,
                   max_len: int = 4096):
    """k requests; each a sorted, de-duplicated list of primes.

    List length = clamp(floor(2**U(0, 12)), 1, max_len) (log-uniform); each
    prime = next_prime(ceil(10**U(log10 lo, log10 hi))), redrawn if >= hi.
    """
    rng = np.random.default_rng(seed)
    lg_lo, lg_hi = math.log10(lo), math.log10(hi)
    reqs = []
    for _ in range(k):
        n = int(min(max(math.floor(2.0 ** rng.uniform(0, 12)), 1), max_len))
        vals = set()
        while len(vals) < n:
            p = next_prime(math.ceil(10.0 ** rng.uniform(lg_lo, lg_hi)))
            if p < hi:
                vals.add(p)
        reqs.append(np.array(sorted(vals), dtype=np.uint64))
    return reqs


def serving_stream(seed: int = 11, n: int = 256, rate: float = 200.0, range_frac: float = 0.5):
    """A finite Poisson stream of queries.

    Each item is a dict: {"t": arrival seconds, "kind": "range"|"prime", ...}.
    Range queries: lo = floor(10**U(6, 10)), len = floor(10**U(3, 6)).
    Single-prime queries: p = next_prime(ceil(10**U(6, 10))).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate)
        if rng.uniform() < range_frac:
            lo = int(10.0 ** rng.uniform(6, 10))
            ln = int(10.0 ** rng.uniform(3, 6))
            out.append({"t": t, "kind": "range", "lo": lo, "hi": lo + ln})
        else:
            p = next_prime(math.ceil(10.0 ** rng.uniform(6, 10)))
            out.append({"t": t, "kind": "prime", "p": p})
    return out
