"""The library's congruence tables (read through the C ABI, host only, no GPU)
checked against the oracle's definitions of B_{p-3}, E_{p-3} mod p for every
prime 11 <= p < 700, and against the costs the paper states for each
congruence (Sec. 2-5).  Transcription slips in an endpoint, a coefficient or a
sign fail one or the other."""
from fractions import Fraction

import pytest

from paper_2101_11157_gb300 import wv
from paper_2101_11157_gb300.workloads import is_prime

# congruence -> (eqn, family, cost / p) as stated in the paper
PAPER = {
    "BB1": ("3.2", 0, Fraction(1, 12)),
    "BB2": ("3.1", 0, Fraction(1, 15)),
    "BB6": ("3.3", 0, Fraction(5, 96)),
    "BB9": ("3.4", 0, Fraction(1, 20)),
    "BB16": ("3.5", 0, Fraction(1, 24)),
    "BB22": ("3.6", 0, Fraction(3, 80)),
    "BB30": ("3.7", 0, Fraction(227, 6480)),
    "EE3": ("5.1", 1, Fraction(3, 16)),
    "EE5": ("5.2", 1, Fraction(9, 64)),
    "EE9": ("5.3", 1, Fraction(43, 384)),
    "EE16": ("5.4", 1, Fraction(205, 2304)),
    "EE24": ("5.5", 1, Fraction(115, 1536)),
    "EE33": ("5.6", 1, Fraction(27, 512)),
}


# generated congruences (greedy search over Prop. 2.1 from BB30 / EE33)
GENERATED = {"BB249": 0, "BB476": 0, "BB1115": 0, "BB2244": 0, "BB3802": 0,
             "EE200": 1, "EE404": 1, "EE967": 1, "EE2004": 1, "EE4122": 1}


def _interval(cid, j):
    import ctypes
    v = [ctypes.c_uint32() for _ in range(4)]
    c = ctypes.c_int64()
    wv.load().wv_congruence_row(cid, j, ctypes.byref(c), *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def tables():
    """name -> (id, kind, lhs, rows); a row is ([(c_k, d_k)], xn, xd, yn, yd)."""
    out = {}
    for cid in range(wv.wv_congruence_count()):
        name, kind, n, lhs = wv.wv_congruence_info(cid)
        rows = [(wv.wv_congruence_terms(cid, j),) + _interval(cid, j) for j in range(n)]
        out[name] = (cid, kind, lhs, rows)
    return out


def _coef(terms, p, e):
    return sum(c * pow(d, -e, p) for c, d in terms) % p


@pytest.fixture(scope="module")
def T():
    return tables()


def test_all_congruences_present(T):
    assert set(T) == set(PAPER) | set(GENERATED)
    assert len(T) == 13 + len(GENERATED)
    assert [T[k][0] for k in sorted(PAPER, key=lambda k: T[k][0])] == list(range(13))
    for name, kind in GENERATED.items():
        assert T[name][1] == kind and len(T[name][3]) == int(name[2:])
    # the paper's rows are plain integers (wv_congruence_row succeeds)
    for name in PAPER:
        assert all(len(r[0]) == 1 and r[0][0][1] == 1 for r in T[name][3])
    assert [len(T[k][3]) for k in ("BB1", "BB2", "BB6", "BB9", "BB16", "BB22", "BB30")] == \
        [1, 2, 6, 9, 16, 22, 30]
    assert [len(T[k][3]) for k in ("EE3", "EE5", "EE9", "EE16", "EE24", "EE33")] == \
        [3, 5, 9, 16, 24, 33]


@pytest.mark.parametrize("name", sorted(PAPER))
def test_cost_matches_paper(T, name):
    cid, kind, lhs, rows = T[name]
    assert kind == PAPER[name][1]
    cost = sum(Fraction(yn, yd) - Fraction(xn, xd) for _, xn, xd, yn, yd in rows)
    assert cost == PAPER[name][2]
    # intervals are disjoint, ascending, inside [0, 1/2], 2,3,5-smooth denominators
    prev = Fraction(0)
    for _, xn, xd, yn, yd in rows:
        x, y = Fraction(xn, xd), Fraction(yn, yd)
        assert prev <= x < y <= Fraction(1, 2)
        prev = y
        for d in (xd, yd):
            for q in (2, 3, 5):
                while d % q == 0:
                    d //= q
            assert d == 1


def _S(p, x, y, e):
    lo = x.numerator * p // x.denominator + 1
    hi = (y.numerator * p + y.denominator - 1) // y.denominator - 1
    return sum(pow(s, -e, p) for s in range(lo, hi + 1)) % p


@pytest.mark.parametrize("name", sorted(GENERATED))
def test_generated_costs_and_intervals(T, name):
    cid, kind, lhs, rows = T[name]
    cost = sum(Fraction(yn, yd) - Fraction(xn, xd) for _, xn, xd, yn, yd in rows)
    # cheaper than the paper's B30 / E33, and cheaper with more sums
    base = PAPER["BB30" if kind == 0 else "EE33"][2]
    assert cost < base
    prev = Fraction(0)
    for terms, xn, xd, yn, yd in rows:
        x, y = Fraction(xn, xd), Fraction(yn, yd)
        assert prev <= x < y <= Fraction(1, 2) and yn < 2**32 and yd < 2**32
        prev = y
        for d in (xd, yd) + tuple(d for _, d in terms):  # subdivisions by d <= 8
            for q in (2, 3, 5, 7):
                while d % q == 0:
                    d //= q
            assert d == 1
    same_kind = sorted((len(T[n][3]), sum(Fraction(r[3], r[4]) - Fraction(r[1], r[2]) for r in T[n][3]))
                       for n, k in GENERATED.items() if k == kind)
    assert all(b[1] < a[1] for a, b in zip(same_kind, same_kind[1:]))


@pytest.mark.parametrize("name", sorted(PAPER) + sorted(GENERATED))
def test_congruence_gives_definition(T, orc, name):
    cid, kind, lhs, rows = T[name]
    e = 3 if kind == 0 else 2
    for p in [p for p in range(11, 700) if is_prime(p)]:
        if lhs % p == 0:
            continue
        rhs = sum(_coef(c, p, e) * _S(p, Fraction(xn, xd), Fraction(yn, yd), e)
                  for c, xn, xd, yn, yd in rows)
        val = rhs * pow(lhs, -1, p) % p
        ref = orc.bernoulli_def(p - 3, p) if kind == 0 else orc.euler_def(p - 3, p)
        assert val == ref, (name, p)


def test_count_terms_matches_rows(T):
    cid_b, cid_e = T["BB30"][0], T["EE33"][0]
    p = 1_062_232_319
    tb, te = wv.wv_count_terms([p], cid_b, cid_e)

    def terms(rows):
        tot = 0
        for _, xn, xd, yn, yd in rows:
            lo = xn * p // xd + 1
            hi = yn * p // yd
            tot += max(0, hi - lo + 1)
        return tot
    assert tb == terms(T["BB30"][3]) and te == terms(T["EE33"][3])
    assert abs(tb / p - 227 / 6480) < 1e-6 and abs(te / p - 27 / 512) < 1e-6


def _inverse_power_prefix(p, e):
    """prefix[s] = sum_{0<i<=s} i^-e mod p for 0 <= s <= (p-1)/2, by Fermat
    inverses in numpy (p < 2^26, so every product fits 64 bits)."""
    import numpy as np
    s = np.arange(1, (p - 1) // 2 + 1, dtype=np.uint64)
    inv, base, k = np.ones_like(s), s.copy(), p - 2
    while k:
        if k & 1:
            inv = inv * base % np.uint64(p)
        base = base * base % np.uint64(p)
        k >>= 1
    t = np.ones_like(s)
    for _ in range(e):
        t = t * inv % np.uint64(p)
    pre = np.zeros(s.size + 1, dtype=np.uint64)
    np.cumsum(t, out=pre[1:])  # < 2^26 * 2^25: no overflow
    return pre % np.uint64(p)


# every row of every generated congruence holds at least one term at the last of these
# (the narrowest rows, of EE2004 and EE4122, need p > 5.88e7)
PRIMES_ALL_ROWS = [12_000_017, 31_000_003, 70_000_027]


@pytest.mark.parametrize("p", PRIMES_ALL_ROWS)
def test_generated_congruences_at_large_primes(T, orc, p):
    """The generated congruences' narrowest rows are empty for every p < 700, so
    the definition test above cannot see a wrong coefficient there.  Each
    congruence, evaluated with exact integers at these primes, must give the
    oracle's B_{p-3} (Stafford-Vandiver, eqn 2.4) and E_{p-3} (Glaisher, eqn
    4.1); at the largest of them every row of every congruence holds at least
    one term, so a wrong coefficient anywhere changes the result."""
    assert is_prime(p)
    want = {0: orc.bernoulli_sv(p), 1: orc.euler_glaisher(p)}
    pre = {3: _inverse_power_prefix(p, 3), 2: _inverse_power_prefix(p, 2)}
    for name in sorted(GENERATED) + ["BB30", "EE33"]:
        cid, kind, lhs, rows = T[name]
        e = 3 if kind == 0 else 2
        rhs, empty = 0, 0
        for terms, xn, xd, yn, yd in rows:
            lo = xn * p // xd + 1                      # first s above x p
            hi = (yn * p + yd - 1) // yd - 1           # last s below y p
            if hi < lo:
                empty += 1
                continue
            S = (int(pre[e][hi]) - int(pre[e][lo - 1])) % p
            rhs += _coef(terms, p, e) * S
        assert rhs * pow(lhs, -1, p) % p == want[kind], (name, p)
        if p == PRIMES_ALL_ROWS[-1]:
            assert empty == 0, (name, p, empty)
