"""Word-level models of the accumulation kernels' modular arithmetic.

The kernels keep values outside [0, p) between reductions (lazy tables,
products not canonicalised) and rely on stated bounds for every word to stay
exact.  These tests replay those routines in Python integers with the same
32- and 64-bit wraparound as the device code (mul.wide / mad.wide, word
packing) and check, on random and extreme inputs, that each result is exact
(no intermediate overflowed), congruent to the intended value mod p, and
inside the bound the next step assumes.  They model csrc/wv_accum.cuh:
the signed 32-bit REDC folded into a wide multiply-add and the per-chain
set-up that uses it (p < 2^30), and the 64-bit path's two-round and
one-round REDC, products, shrink and set-up (2^31 <= p < 2^37).  No GPU
is involved; the GPU parity tests check the kernels' residues themselves."""
import random

import pytest

M32, M64 = 1 << 32, 1 << 64


def s32(v):
    v %= M32
    return v - M32 if v >= 1 << 31 else v


def s64(v):
    v %= M64
    return v - M64 if v >= 1 << 63 else v


def odd_moduli(rng, lo, hi, k):
    out = [lo | 1, (hi - 1) | 1 if ((hi - 1) | 1) < hi else hi - 2]
    while len(out) < k:
        out.append(rng.randrange(lo, hi) | 1)
    return [p for p in out if lo <= p < hi]


# ---------------------------------------------------------------- 32-bit path
def sredc(a, b, p):
    """hi32(mad.wide(lo32(w) * q, -p, w)) with w = mul.wide(a, b), q = p^-1 mod 2^32."""
    q = pow(p, -1, M32)
    w = s64(a * b)
    assert w == a * b  # mul.wide of two int32 is exact
    m = s32((w % M32) * q)
    d = s64(w + m * s32(-p))
    assert d == w - m * p and d % M32 == 0
    return s32(d >> 32)


def sredc_sum(w, p):
    """hi32(mad.wide(lo32(w) * q, -p, w)) for a 64-bit sum w of products."""
    q = pow(p, -1, M32)
    assert s64(w) == w
    m = s32((w % M32) * q)
    d = s64(w + m * s32(-p))
    assert d == w - m * p and d % M32 == 0
    return s32(d >> 32)


@pytest.mark.parametrize("seed", [1, 2])
def test_signed_redc_value_and_bound(seed):
    """REDC of w = a b is a b 2^-32 mod p and lies within |w| / 2^32 + p / 2."""
    rng = random.Random(seed)
    for p in odd_moduli(rng, 3, 1 << 30, 40):
        r32inv = pow(M32, -1, p)
        for _ in range(50):
            a = rng.randrange(-(1 << 31), 1 << 31)
            b = rng.randrange(-(1 << 31), 1 << 31)
            if abs(a * b) >= 1 << 62:
                continue
            r = sredc(a, b, p)
            assert (r - a * b * r32inv) % p == 0
            assert abs(r) <= abs(a * b) / M32 + p / 2


def test_uform_powers_signed_range():
    """From u in [0, p) (p < 2^30): u u 2^-32 in (-3p/4, 3p/4), u^3 2^-64 in (-p, p)."""
    rng = random.Random(3)
    for p in odd_moduli(rng, 1 << 20, 1 << 30, 30) + [(1 << 30) - 35]:
        for u in [0, 1, p - 1, p // 2] + [rng.randrange(p) for _ in range(60)]:
            u2 = sredc(u, u, p)
            assert abs(u2) < 3 * p / 4
            assert abs(sredc(u2, u, p)) < p


@pytest.mark.parametrize("K,ex", [(4, 3), (6, 2), (8, 3), (10, 2)])
def test_chain_setup_signed_bounds(K, ex):
    """The set-up of one point on the signed path: from t in [0, p) and u's
    factor x falling by one a term from [0, p) (at most 2^10 below 0), the
    products P, Pu stay in (-p, p) and Q = REDC(Q t) + P in (-2p, 2p), so one
    correction per point gives the canonical values of the canonical
    recurrence."""
    rng = random.Random(K * 10 + ex)
    for p in odd_moduli(rng, 11, 1 << 30, 25) + [11, 101, (1 << 30) - 35]:
        r32inv = pow(M32, -1, p)
        one = M32 % p
        for _ in range(20):
            ts = [rng.randrange(p) for _ in range(K)]
            # a later point's x may already lie below 0 (by up to K (DTOP + 1) < 2^10)
            x = rng.randrange(p) if rng.random() < 0.7 else rng.randrange(-1000, min(p, 64))
            xs = [x - i for i in range(K)]
            P = Q = Pu = None
            cP = cQ = cPu = None  # the canonical recurrence mod p
            for i, t in enumerate(ts):
                if i == 0:
                    P, Q, Pu = t, one, xs[0]
                    cP, cQ, cPu = t % p, one, xs[0] % p
                else:
                    Q = sredc(Q, t, p) + P
                    P = sredc(P, t, p)
                    Pu = sredc(Pu, xs[i], p)
                    cQ = (cQ * t * r32inv + cP) % p
                    cP = cP * t * r32inv % p
                    cPu = cPu * xs[i] * r32inv % p
                assert abs(P) < p and abs(Q) < 2 * p and -(1 << 31) <= Q < 1 << 31
                assert i == 0 or abs(Pu) < p
            assert (P % p, Q % p, Pu % p) == (cP, cQ, cPu)


# ---------------------------------------------------------------- 64-bit path
def lo(v):
    return v % M32


def hi(v):
    return (v >> 32) % M32


def umad(a, b, c):
    assert 0 <= a < M32 and 0 <= b < M32 and 0 <= c < M64
    return (a * b + c) % M64


def upack(l, h):
    return (h % M32) * M32 + l % M32


class K64:
    def __init__(self, p):
        self.p, self.p0, self.p1 = p, lo(p), hi(p)
        self.q = (-pow(p, -1, M32)) % M32
        self.mhi = (1 << 62) // p
        np_ = (M64 - p) % M64
        self.np0, self.np1 = lo(np_), hi(np_)


def m64_prod(c, g):
    c0, c1, g0, g1 = lo(c), hi(c), lo(g), hi(g)
    X = umad(c0, g0, 0)
    Y = umad(c0, g1, hi(X))
    Y = umad(c1, g0, Y)
    return lo(X), upack(lo(Y), hi(Y) + c1 * g1)


def m64_prod2(ca, ga, cb, gb):
    a0, a1, x0, x1 = lo(ca), hi(ca), lo(ga), hi(ga)
    b0, b1, y0, y1 = lo(cb), hi(cb), lo(gb), hi(gb)
    Xa = umad(a0, x0, 0)
    Xb = umad(b0, y0, lo(Xa))
    Y = umad(a0, x1, hi(Xa))
    Y = umad(a1, x0, Y)
    Y = umad(b0, y1, Y)
    Y = (umad(b1, y0, Y) + hi(Xb)) % M64
    return lo(Xb), upack(lo(Y), hi(Y) + a1 * x1 + b1 * y1)


def m64_redc2(T0, TY, k):
    m0 = T0 * k.q % M32
    A = umad(m0, k.p0, T0)
    U = (umad(m0, k.p1, TY) + hi(A)) % M64
    m1 = lo(U) * k.q % M32
    B = umad(m1, k.p0, lo(U))
    return (umad(m1, k.p1, hi(U)) + hi(B)) % M64


def m64_redc1(T0, TY, k):
    m0 = T0 * k.q % M32
    A = umad(m0, k.p0, T0)
    return (umad(m0, k.p1, TY) + hi(A)) % M64


def m64_shrink_q(v, k):
    qq = ((hi(v) << 2) % M32) * k.mhi >> 32
    r = umad(qq, k.np0, v)
    return upack(lo(r), hi(r) + qq * k.np1)


def checked_prod(c, g):
    T0, TY = m64_prod(c, g)
    assert T0 + TY * M32 == c * g  # no word overflowed
    return T0, TY


def primes64(rng, k):
    return odd_moduli(rng, 1 << 31, 1 << 37, k) + [(1 << 37) - 25, (1 << 31) + 11]


def test_m64_redc_rounds_value_and_bound():
    """Two rounds give T 2^-64 mod p below T / 2^64 + p; one round gives
    T 2^-32 mod p below T / 2^32 + p, exactly (T < 2^96)."""
    rng = random.Random(5)
    for p in primes64(rng, 20):
        k = K64(p)
        for _ in range(40):
            T = rng.randrange(1 << rng.choice([64, 80, 95]))
            T0, TY = T % M32, T >> 32
            r2 = m64_redc2(T0, TY, k)
            assert (r2 * M64 - T) % p == 0 and r2 < T / M64 + p
            r1 = m64_redc1(T0, TY, k)
            assert (r1 * M32 - T) % p == 0 and r1 < T / M32 + p


def test_m64_shrink_below_6p():
    rng = random.Random(6)
    for p in primes64(rng, 20):
        k = K64(p)
        for v in [0, (1 << 58) - 1] + [rng.randrange(1 << 58) for _ in range(50)]:
            r = m64_shrink_q(v, k)
            assert r % p == v % p and r < 6 * p


def test_m64_uform_one_round_products_stay_in_bounds():
    """u's lazy value shrunk below 6p; u u 2^-32 < 2^47.2 and u^3 2^-64 < 2^55
    (both below 2^57); the pair update c0 A and c1 A + c0 G1 (c0, c1 below
    p + 2^32, G1 below 2^57) stays below 2^96 and exact, and its two-round
    results stay below p + 2^32."""
    rng = random.Random(7)
    for p in primes64(rng, 16):
        k = K64(p)
        for _ in range(30):
            v = rng.choice([(1 << 57) - 1, rng.randrange(1 << 57)])
            Us = m64_shrink_q(v, k)
            if rng.random() < 0.2:
                Us = 6 * p - 1  # the bound itself
            A1 = m64_redc1(*checked_prod(Us, Us), k)
            assert A1 < 2 ** 47.2
            A = m64_redc1(*checked_prod(A1, Us), k)
            assert A < 2 ** 55
            assert (A * M64 - Us ** 3) % p == 0
            for A_ in (A1, A):  # squares use A1, cubes A
                c0 = rng.choice([p + M32 - 1, rng.randrange(p + M32)])
                c1 = rng.choice([p + M32 - 1, rng.randrange(p + M32)])
                g1 = rng.choice([(1 << 57) - 1, rng.randrange(1 << 57)])
                T0, TY = checked_prod(c0, A_)
                n0 = m64_redc2(T0, TY, k)
                T0, TY = m64_prod2(c1, A_, c0, g1)
                assert T0 + TY * M32 == c1 * A_ + c0 * g1 < 1 << 96
                n1 = m64_redc2(T0, TY, k)
                assert n0 < p + M32 and n1 < p + M32


@pytest.mark.parametrize("K", [8, 12, 16])
def test_m64_setup_products_without_canonicalisation(K):
    """The 64-bit set-up: products of inputs below about 2^38 stay below
    p + 2^12, so P, Pu < p + 2^12 and Q = REDC2(Q t) + P < 2p + 2^13 over a
    point's K terms, with u's factor kept as x + p (it falls by at most
    2^10); two conditional subtractions make Q canonical."""
    rng = random.Random(K)
    for p in primes64(rng, 12):
        k = K64(p)
        one = M64 % p
        for _ in range(10):
            ts = [rng.randrange(p) for _ in range(K)]
            x = rng.randrange(p) + p
            P = Q = Pu = None
            for i, t in enumerate(ts):
                if i == 0:
                    P, Q, Pu = t, one, x
                else:
                    Q = m64_redc2(*checked_prod(Q, t), k) + P
                    P = m64_redc2(*checked_prod(P, t), k)
                    Pu = m64_redc2(*checked_prod(Pu, x - i), k)
                    assert P < p + (1 << 12) and Pu < p + (1 << 12)
                assert Q < 2 * p + (1 << 13) and Q < 2 ** 38.01
            qc = Q - p if Q >= p else Q
            qc = qc - p if qc >= p else qc
            assert 0 <= qc < p and qc == Q % p


# ------------------------------------------------------ one chain, mod p
def chain_model(s, n, K, ex, p, R, uf, half=False):
    """The grouped chain of tile_m31_grouped / tile_m64_grouped modelled mod p,
    each REDC as a factor R^-1 (or h^-1 = 2^-32 for the 64-bit u form's
    one-round products, `half`): tables from the set-up points (top down,
    folded into the diagonals over their whole length, odd orders negated),
    stepped by additions; each group's tabled values are checked against the
    group's own products; returns c1 / c0 after the groups, the scale and
    the single-term tail."""
    Ri = pow(R, -1, p)
    hi_ = pow(1 << 32, -1, p)
    DA, DB = K * ex, (K - 1) * ex
    DT = K if uf else DA
    DTOP = max(DT, DB)
    one = R % p

    def point(m):  # the K consecutive x of point m, from the top down
        xs = [s + m * K + K - 1 - i for i in range(K)]
        ts = [pow(x, ex, p) for x in xs]
        P, Q, Pu = ts[0], one, xs[0] % p
        for i in range(1, K):
            Q = (Q * ts[i] * Ri + P) % p
            P = P * ts[i] * Ri % p
            Pu = Pu * xs[i] * Ri % p
        return P, Q, Pu

    va, vb = [0] * (DT + 1), [0] * (DB + 1)
    for m in range(DTOP, -1, -1):
        P, Q, Pu = point(m)
        for vals, nv, D in ((va, Pu if uf else P, DT), (vb, Q, DB)):
            if m > D:
                continue
            for j in range(D + 1):
                old = vals[j]
                vals[j] = nv
                if j < D:
                    nv = (nv - old) % p
    ga = [(-v) % p if j & 1 else v for j, v in enumerate(va)]
    gb = [(-v) % p if j & 1 else v for j, v in enumerate(vb)]
    G = n // K
    c0, c1 = one, 0
    for g in range(G):
        P, Q, Pu = point(g)
        assert ga[0] == (Pu if uf else P) and gb[0] == Q, g  # the tables reproduce the group
        A = ga[0]
        if uf:
            u = A
            if half:  # one-round products: u u 2^-32 (u^3 2^-64)
                A = u * u * hi_ % p
                if ex == 3:
                    A = A * u * hi_ % p
            else:
                A = u * u * Ri % p
                if ex == 3:
                    A = A * u * Ri % p
        c0, c1 = c0 * A * Ri % p, (c1 * A + c0 * gb[0]) * Ri % p
        for tab in (ga, gb):
            for j in range(len(tab) - 1):
                tab[j] = (tab[j] + tab[j + 1]) % p
    if uf:
        if half:  # (ex - 1)(2K - 1) one-round steps of f = R, then c1 f R^-1
            f = one
            for _ in range((ex - 1) * (2 * K - 1)):
                f = f * hi_ % p
        else:  # (ex - 1) K steps f <- f 1 R^-1
            f = one
            for _ in range((ex - 1) * K):
                f = f * Ri % p
        c1 = c1 * f * Ri % p
    for x in range(s + G * K, s + n):  # the tail, one term at a time (eqn 3.12)
        t = pow(x, ex, p)
        c0, c1 = c0 * t * Ri % p, (c1 * t * Ri + c0) % p
    return c1 * pow(c0, -1, p) % p


@pytest.mark.parametrize("K,ex,uf,half", [(2, 3, False, False), (3, 2, False, False),
                                          (4, 3, False, False), (8, 3, True, False),
                                          (10, 2, True, False), (12, 3, True, True),
                                          (16, 2, True, True), (8, 3, True, True)])
def test_chain_model_equals_single_terms(K, ex, uf, half):
    """Groups of K terms through the difference tables give c1 / c0 = R sum
    s^-e, as single-term steps do (eqn 3.12 against eqn 3.14), for the pair
    tables, the u form and the 64-bit u form's one-round products."""
    rng = random.Random(K * 7 + ex)
    R = 1 << (64 if half else 32)
    for p in (1000003, 1062232319, 2147483647, 99999998237):
        if not half and p >= 1 << 31:
            continue
        for _ in range(3):
            n = rng.randrange(K * (K * ex + 2), K * (K * ex + 2) + 3 * K)
            s = rng.randrange(1, p - n - 1)
            want = R * sum(pow(pow(x, ex, p), -1, p) for x in range(s, s + n)) % p
            assert chain_model(s, n, K, ex, p, R, uf, half) == want


def test_pair_update_signed_keeps_accumulators_in_range():
    """The signed path's group step c0 <- REDC(c0 G0), c1 <- REDC(c1 G0 + c0 G1)
    (p < 2^30): with G0 in (-p, p) (a u-form power, or a canonical table
    value) and G1 in [0, p), c0 and c1 stay in (-p, p) group after group,
    every wide product exact, and the pair stays correct mod p."""
    rng = random.Random(11)
    for p in odd_moduli(rng, 3, 1 << 30, 12) + [(1 << 30) - 35, 1062232319 % (1 << 30) | 1]:
        Ri = pow(M32, -1, p)
        c0, c1 = M32 % p, 0
        e0, e1 = c0, c1
        for _ in range(300):
            A = rng.choice([rng.randrange(-p + 1, p), p - 1, -p + 1, 0])
            B = rng.choice([rng.randrange(p), p - 1])
            w1 = c1 * A + c0 * B  # mad.wide(c0, B, mul.wide(c1, A))
            assert abs(w1) < 1 << 63
            c0, c1 = sredc(c0, A, p), sredc_sum(w1, p)
            e0, e1 = e0 * A * Ri % p, (e1 * A + e0 * B) * Ri % p
            assert abs(c0) < p and abs(c1) < p
            assert (c0 - e0) % p == 0 and (c1 - e1) % p == 0


def test_pair_update_unsigned_canonical():
    """2^30 <= p < 2^31 (unsigned words): c0 G0 and c1 G0 + c0 G1 stay below
    2 p^2 < 2^63, the REDC's high word below 2p, and one conditional
    subtraction makes each result canonical."""
    rng = random.Random(12)
    for p in odd_moduli(rng, 1 << 30, 1 << 31, 12) + [2147483647]:
        qn = (-pow(p, -1, M32)) % M32
        Ri = pow(M32, -1, p)

        def redc(w):
            assert 0 <= w < 1 << 63
            m = lo(w) * qn % M32
            t = hi(umad(m, p, w))
            return min(t, (t - p) % M32)

        c0, c1 = M32 % p, 0
        for _ in range(300):
            A, B = rng.randrange(p), rng.randrange(p)
            w0, w1 = c0 * A, c1 * A + c0 * B
            assert w1 < 2 * p * p < 1 << 63
            n0, n1 = redc(w0), redc(w1)
            assert n0 == w0 * Ri % p and n1 == w1 * Ri % p
            c0, c1 = n0, n1
