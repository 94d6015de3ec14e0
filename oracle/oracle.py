"""Python face of the plain CPU oracle (``wv_oracle.c``) plus exact rational
Bernoulli/Euler numbers.

TEST INFRASTRUCTURE ONLY: the product package never imports this module.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path.

Levels (see ``wv_oracle.c`` for the passage each one follows):

* ``exact_bernoulli`` / ``exact_euler`` -- exact rationals/integers from the
  generating functions of Sec. 1 (pure Python, small n).
* ``bernoulli_def`` / ``euler_def`` -- the same recurrences reduced mod p in C
  (O(p^2)).
* ``bernoulli_glaisher`` (eqn 1.2), ``bernoulli_h2`` (eqn 1.1),
  ``wolstenholme_bits`` (eqn 1.1 literally).
* ``bernoulli_sv`` (eqn 2.4 -> eqn 3.2), ``bernoulli_v12`` (eqn 2.8),
  ``euler_glaisher`` (eqn 4.1, sign (-1)^k), ``euler_mcintosh`` (eqn 4.7).
* ``bernoulli_pm3`` / ``euler_pm3`` / ``residues`` -- the default large-p pair
  (Stafford-Vandiver for B, Glaisher for E), threaded over primes.
* ``sieve`` -- plain sieve of Eratosthenes on a window.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from fractions import Fraction
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

U64_MAX = (1 << 64) - 1

METHOD_B = {"default": 0, "def": 1, "h2": 2, "glaisher": 3, "sv": 4, "v12": 5}
METHOD_E = {"default": 0, "def": 1, "glaisher": 6, "mcintosh": 7}


def build(force: bool = False) -> str:
    """Compile ``wv_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, i32 = ctypes.c_uint64, ctypes.c_int
        p64 = ctypes.POINTER(ctypes.c_uint64)
        for name, args in [
            ("orc_bernoulli_def", [u64, u64]), ("orc_euler_def", [u64, u64]),
            ("orc_bernoulli_glaisher", [u64, u64]), ("orc_bernoulli_h2", [u64]),
            ("orc_bernoulli_sv", [u64]), ("orc_bernoulli_v12", [u64]),
            ("orc_euler_glaisher", [u64]), ("orc_euler_mcintosh", [u64]),
            ("orc_bernoulli_pm3", [u64]), ("orc_euler_pm3", [u64]),
            ("orc_mulmod", [u64, u64, u64]), ("orc_powmod", [u64, u64, u64]),
            ("orc_invmod", [u64, u64]),
            ("orc_interval_sum", [u64, u64, u64, u64, u64, ctypes.c_uint, i32]),
            ("orc_sieve", [u64, u64, p64, u64]),
        ]:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = u64
        lib.orc_wolstenholme_bits.argtypes = [u64]
        lib.orc_wolstenholme_bits.restype = i32
        lib.orc_residues.argtypes = [p64, ctypes.c_size_t, p64, p64, i32, i32, i32]
        lib.orc_residues.restype = i32
        _lib = lib
        return lib


def _chk(v: int) -> int:
    if v == U64_MAX:
        raise ValueError("oracle: argument outside the formula's range of validity")
    return int(v)


# --------------------------------------------------------------------------
# exact rationals (Sec. 1 generating functions), pure Python
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def _bernoulli_list(n: int) -> tuple:
    """B_0..B_n from sum_{j=0}^{m} C(m+1, j) B_j = 0 (m >= 1)."""
    from math import comb
    B = [Fraction(1)]
    for m in range(1, n + 1):
        acc = sum(comb(m + 1, j) * B[j] for j in range(m))
        B.append(-acc / (m + 1))
    return tuple(B)


@lru_cache(maxsize=None)
def _euler_list(n: int) -> tuple:
    """E_0..E_n (sec convention) from sum_j (-1)^j C(m, 2j) E_{m-2j} = 0."""
    from math import comb
    E = [1] + [0] * n
    for m in range(2, n + 1, 2):
        E[m] = -sum((-1) ** j * comb(m, 2 * j) * E[m - 2 * j] for j in range(1, m // 2 + 1))
    return tuple(E)


def exact_bernoulli(n: int) -> Fraction:
    return _bernoulli_list(n)[n]


def exact_euler(n: int) -> int:
    return _euler_list(n)[n]


def rational_mod(x: Fraction, p: int) -> int:
    """num * den^-1 mod p (p must not divide the denominator)."""
    if x.denominator % p == 0:
        raise ZeroDivisionError(f"{p} divides the denominator of {x}")
    return x.numerator * pow(x.denominator, -1, p) % p


# --------------------------------------------------------------------------
# C oracle wrappers
# --------------------------------------------------------------------------
def bernoulli_def(n: int, p: int) -> int:
    return _chk(_load().orc_bernoulli_def(n, p))


def euler_def(n: int, p: int) -> int:
    return _chk(_load().orc_euler_def(n, p))


def bernoulli_glaisher(p: int, h: int = 2) -> int:
    return _chk(_load().orc_bernoulli_glaisher(p, h))


def bernoulli_h2(p: int) -> int:
    return _chk(_load().orc_bernoulli_h2(p))


def wolstenholme_bits(p: int) -> int:
    return int(_load().orc_wolstenholme_bits(p))


def bernoulli_sv(p: int) -> int:
    return _chk(_load().orc_bernoulli_sv(p))


def bernoulli_v12(p: int) -> int:
    return _chk(_load().orc_bernoulli_v12(p))


def euler_glaisher(p: int) -> int:
    return _chk(_load().orc_euler_glaisher(p))


def euler_mcintosh(p: int) -> int:
    return _chk(_load().orc_euler_mcintosh(p))


def bernoulli_pm3(p: int) -> int:
    return _chk(_load().orc_bernoulli_pm3(p))


def euler_pm3(p: int) -> int:
    return _chk(_load().orc_euler_pm3(p))


def interval_sum(p: int, x: Fraction, y: Fraction, e: int, alternating: bool = False) -> int:
    """sum_{xp<s<yp} (+-1)^s s^-e mod p (eqn 2.3 / eqn 4.7's S~)."""
    x, y = Fraction(x), Fraction(y)
    return _chk(_load().orc_interval_sum(p, x.numerator, x.denominator, y.numerator,
                                         y.denominator, e, int(alternating)))


def residues(primes, method_b: str | None = "default", method_e: str | None = "default",
             threads: int | None = None):
    """(B_{p-3} mod p, E_{p-3} mod p) arrays for a list of primes, threaded.

    Either method may be None to skip that residue.  Returns numpy uint64
    arrays (or None for a skipped one)."""
    lib = _load()
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
    n = pr.size
    ob = np.zeros(n, dtype=np.uint64) if method_b is not None else None
    oe = np.zeros(n, dtype=np.uint64) if method_e is not None else None
    ptr = lambda a: (a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if a is not None
                     else ctypes.POINTER(ctypes.c_uint64)())
    if threads is None:
        threads = os.cpu_count() or 1
    lib.orc_residues(ptr(pr), n, ptr(ob), ptr(oe),
                     METHOD_B[method_b] if method_b is not None else 0,
                     METHOD_E[method_e] if method_e is not None else 0, int(threads))
    for a in (ob, oe):
        if a is not None and n and np.any(a == np.uint64(U64_MAX)):
            raise ValueError("oracle: a prime outside the chosen formula's validity range")
    return ob, oe


def sieve(lo: int, hi: int) -> np.ndarray:
    """All primes in [lo, hi), ascending, as uint64."""
    lib = _load()
    n = int(lib.orc_sieve(lo, hi, ctypes.POINTER(ctypes.c_uint64)(), 0))
    if n == U64_MAX:
        raise MemoryError("oracle sieve: window too large")
    out = np.zeros(max(n, 1), dtype=np.uint64)
    lib.orc_sieve(lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n)
    return out[:n]


def symmetric(r: int, p: int) -> int:
    """The representative of r mod p in (-p/2, p/2] (Sec. 3, near-miss tables)."""
    r %= p
    return r - p if r > p // 2 else r


def histogram(primes, residues, bins: int = 2000) -> np.ndarray:
    """Counts of <r>_p / p over `bins` equal bins of (-1/2, 1/2] (Sec. 3
    "Results": the 2000-bin histogram of <B_{p-3}>_p / p).  Bin b holds the
    primes with u = <r>_p / p + 1/2 in [b / bins, (b + 1) / bins), computed
    with exact rationals."""
    out = np.zeros(bins, dtype=np.int64)
    for p, r in zip(primes, residues):
        p, r = int(p), int(r)
        u = Fraction(symmetric(r, p), p) + Fraction(1, 2)
        out[math.floor(u * bins)] += 1
    return out


def bernoulli_general(p: int, e: int) -> int:
    """B_{p-e} mod p for odd e >= 3 and p >= e + 3 (-1 where the congruence's
    constant vanishes mod p), by the Stafford-Vandiver congruence (Sec. 2,
    eqn 2.4) in its general form: C_k(3,4,6) B_{2k} = S_{2k-1}(1/6, 1/4) with
    2k = p - e and C_k(a,b,c) = (a^{p-2k} + b^{p-2k} - c^{p-2k} - 1) / (4k).
    The sum has exponent 2k - 1 = p - 1 - e, i.e. the inverse powers s^-e."""
    two_k = p - e
    c = (pow(3, e, p) + pow(4, e, p) - pow(6, e, p) - 1) * pow(2 * two_k, -1, p) % p
    if c == 0:
        return -1
    return interval_sum(p, Fraction(1, 6), Fraction(1, 4), e) * pow(c, -1, p) % p


def euler_general(p: int, e: int) -> int:
    """E_{p-1-e} mod p for even e >= 2 and p >= e + 3, by Glaisher's congruence
    (Sec. 4, eqn 4.1, with the sign (-1)^k): (-1)^k 4^{2k-1} E_{p-1-2k} =
    S_{p-1-2k}(0, 1/4) with 2k = e, the sum of the inverse powers s^-e."""
    k = e // 2
    lhs = (-1) ** k * pow(4, 2 * k - 1, p) % p
    return interval_sum(p, Fraction(0), Fraction(1, 4), e) * pow(lhs, -1, p) % p
