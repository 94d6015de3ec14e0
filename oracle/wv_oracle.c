/*
 * wv_oracle.c -- plain CPU oracle for B_{p-3} mod p and E_{p-3} mod p.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * Everything here is deliberately simple: 128-bit products reduced with `%`,
 * loops in the order the mathematics states them, no blocking or reordering.
 *
 * Three levels, each citing the passage it follows:
 *   A  definitions (O(p^2)): B_n from the generating function z/(e^z-1)
 *      (Sec. 1, definition of B_k) and E_n from sec z (Sec. 1, definition of
 *      E_k, sec convention of the footnote), both reduced mod p.
 *   B  classical closed forms for B_{p-3}: Glaisher's binomial congruence
 *      (Sec. 1, eqn 1.2) and the harmonic sum of eqn 1.1 (sum k^-2 mod p^2).
 *   C  single-sum classical congruences specialised to k=(p-3)/2 (Sec. 3)
 *      and k=1 (Sec. 5), each evaluated with the polynomial accumulation of
 *      eqn 3.12:  Stafford-Vandiver (eqn 2.4 -> BB1), Voronoi (eqn 2.8),
 *      Glaisher's Euler congruence (eqn 4.1, sign as read below) and
 *      McIntosh's alternating congruence (eqn 4.7).
 *
 * Reading of eqn 4.1: the printed sign factor (-1)^{(p-1)/2-k} does not
 * match the definition for p = 3 mod 4; the factor (-1)^k, the one carried
 * by every congruence derived from it (eqns 4.2-4.6), is used.  At k = 1
 * this is  -4 E_{p-3} = sum_{0<s<p/4} s^-2  (mod p).
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* modular helpers (any modulus m < 2^64)                              */
/* ------------------------------------------------------------------ */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((u128)a * b) % m);
}
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((u128)(a % m) + (b % m)) % m);
}
static uint64_t submod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((u128)(a % m) + m - (b % m)) % m);
}
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}
/* inverse of a modulo m (gcd(a,m)=1) by the extended Euclidean algorithm */
static uint64_t invmod(uint64_t a, uint64_t m) {
    __int128 t = 0, newt = 1;
    __int128 r = m, newr = a % m;
    while (newr != 0) {
        __int128 q = r / newr, tmp;
        tmp = t - q * newt; t = newt; newt = tmp;
        tmp = r - q * newr; r = newr; newr = tmp;
    }
    if (r != 1) return 0; /* not invertible */
    if (t < 0) t += m;
    return (uint64_t)t;
}
/* signed integer c reduced into [0,m) */
static uint64_t smod(int64_t c, uint64_t m) {
    __int128 r = (__int128)c % (__int128)m;
    if (r < 0) r += m;
    return (uint64_t)r;
}

uint64_t orc_mulmod(uint64_t a, uint64_t b, uint64_t m) { return mulmod(a, b, m); }
uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t m) { return powmod(a, e, m); }
uint64_t orc_invmod(uint64_t a, uint64_t m) { return invmod(a, m); }

/* ------------------------------------------------------------------ */
/* Level A: definitions                                                */
/* ------------------------------------------------------------------ */

/* Factorials and inverse factorials mod p for 0..n (n < p). */
static int fact_tables(uint64_t n, uint64_t p, uint64_t **f, uint64_t **fi) {
    *f = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    *fi = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    if (!*f || !*fi) { free(*f); free(*fi); return -1; }
    (*f)[0] = 1 % p;
    for (uint64_t i = 1; i <= n; ++i) (*f)[i] = mulmod((*f)[i - 1], i, p);
    for (uint64_t i = 0; i <= n; ++i) (*fi)[i] = invmod((*f)[i], p);
    return 0;
}
static uint64_t binom_p(uint64_t n, uint64_t k, uint64_t p,
                        const uint64_t *f, const uint64_t *fi) {
    if (k > n) return 0;
    return mulmod(mulmod(f[n], fi[k], p), fi[n - k], p);
}

/*
 * B_n mod p from the generating function z/(e^z - 1) = sum B_k z^k/k!
 * (Sec. 1).  Multiplying by (e^z - 1)/z = sum z^j/(j+1)! and comparing the
 * coefficient of z^n gives, for n >= 1,  sum_{j=0}^{n} C(n+1, j) B_j = 0,
 * i.e.  B_n = -(1/(n+1)) sum_{j<n} C(n+1, j) B_j.
 * Needs n + 1 < p so every factorial is a unit mod p.  Returns UINT64_MAX on
 * bad arguments.  Cost O(n^2).
 */
uint64_t orc_bernoulli_def(uint64_t n, uint64_t p) {
    if (p < 3 || n + 1 >= p) return UINT64_MAX;
    uint64_t *f, *fi;
    if (fact_tables(n + 1, p, &f, &fi)) return UINT64_MAX;
    uint64_t *B = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    B[0] = 1 % p;
    for (uint64_t m = 1; m <= n; ++m) {
        uint64_t acc = 0;
        for (uint64_t j = 0; j < m; ++j)
            acc = addmod(acc, mulmod(binom_p(m + 1, j, p, f, fi), B[j], p), p);
        /* (m+1) B_m = -acc */
        B[m] = mulmod(submod(0, acc, p), invmod((m + 1) % p, p), p);
    }
    uint64_t r = B[n];
    free(B); free(f); free(fi);
    return r;
}

/*
 * E_n mod p from sec z = sum E_k z^k/k! (Sec. 1, sec convention).
 * sec z * cos z = 1 gives, for even n >= 2,
 *   sum_{j=0}^{n/2} (-1)^j C(n, 2j) E_{n-2j} = 0,
 * i.e.  E_n = -sum_{j=1}^{n/2} (-1)^j C(n, 2j) E_{n-2j};  odd E_n = 0.
 * Needs n < p.  Cost O(n^2).
 */
uint64_t orc_euler_def(uint64_t n, uint64_t p) {
    if (p < 3 || n >= p) return UINT64_MAX;
    if (n & 1) return 0;
    uint64_t *f, *fi;
    if (fact_tables(n, p, &f, &fi)) return UINT64_MAX;
    uint64_t *E = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    E[0] = 1 % p;
    for (uint64_t m = 2; m <= n; m += 2) {
        uint64_t acc = 0; /* sum_{j=1}^{m/2} (-1)^j C(m,2j) E_{m-2j} */
        for (uint64_t j = 1; 2 * j <= m; ++j) {
            uint64_t term = mulmod(binom_p(m, 2 * j, p, f, fi), E[m - 2 * j], p);
            acc = (j & 1) ? submod(acc, term, p) : addmod(acc, term, p);
        }
        E[m] = submod(0, acc, p);
    }
    uint64_t r = E[n];
    free(E); free(f); free(fi);
    return r;
}

/* ------------------------------------------------------------------ */
/* Level B: classical closed forms for B_{p-3}                         */
/* ------------------------------------------------------------------ */

/*
 * Glaisher (Sec. 1, eqn 1.2):  C(hp-1, p-1) = 1 - h(h-1)/3 p^3 B_{p-3} mod p^4.
 * C(hp-1, p-1) = prod_{k=1}^{p-1} (hp - k)/k, evaluated mod p^4 (the
 * denominator (p-1)! is a unit).  Then
 *   B_{p-3} = -3 ((C - 1)/p^3) / (h(h-1))  mod p.
 * Needs p^4 < 2^64 (p < 65536), p >= 5, 2 <= h.  Returns UINT64_MAX otherwise.
 */
uint64_t orc_bernoulli_glaisher(uint64_t p, uint64_t h) {
    if (p < 5 || p >= 65536 || h < 2 || h % p == 0 || (h - 1) % p == 0) return UINT64_MAX;
    uint64_t m = p * p * p * p;
    uint64_t num = 1 % m, den = 1 % m;
    for (uint64_t k = 1; k < p; ++k) {
        num = mulmod(num, (h * p - k) % m, m);
        den = mulmod(den, k, m);
    }
    uint64_t c = mulmod(num, invmod(den, m), m);
    uint64_t cm1 = submod(c, 1, m);
    uint64_t p3 = p * p * p;
    if (cm1 % p3 != 0) return UINT64_MAX; /* Wolstenholme's theorem violated */
    uint64_t q = (cm1 / p3) % p;
    uint64_t hh = mulmod(h % p, (h - 1) % p, p);
    /* B = -3 q / (h(h-1)) */
    return mulmod(submod(0, mulmod(3, q, p), p), invmod(hh, p), p);
}

/*
 * Harmonic form (Sec. 1, eqn 1.1 and the classical congruence behind it):
 *   H2 = sum_{0<k<p} k^-2 = (2/3) p B_{p-3}  (mod p^2),
 * so p is a Wolstenholme prime exactly when H2 = 0 mod p^2.
 * H2 is accumulated as a fraction N/D mod p^2 (N <- N k^2 + D, D <- D k^2)
 * and B_{p-3} = (3/2) (H2 / p) mod p.  Needs p < 2^32.
 */
uint64_t orc_bernoulli_h2(uint64_t p) {
    if (p < 5 || p >= (1ull << 32)) return UINT64_MAX;
    uint64_t m = p * p;
    uint64_t N = 0, D = 1;
    for (uint64_t k = 1; k < p; ++k) {
        uint64_t k2 = mulmod(k, k, m);
        N = addmod(mulmod(N, k2, m), D, m);
        D = mulmod(D, k2, m);
    }
    uint64_t H2 = mulmod(N, invmod(D, m), m);
    if (H2 % p != 0) return UINT64_MAX; /* Wolstenholme's theorem violated */
    uint64_t h = (H2 / p) % p;
    return mulmod(mulmod(3, h, p), invmod(2, p), p);
}

/*
 * The three congruences of eqn 1.1 evaluated literally (tiny p only,
 * p^4 < 2^64): bit0  sum k^-2 = 0 mod p^2,  bit1  sum k^-1 = 0 mod p^3,
 * bit2  C(2p-1,p-1) = 1 mod p^4.
 */
int orc_wolstenholme_bits(uint64_t p) {
    if (p < 5 || p >= 65536) return -1;
    int bits = 0;
    uint64_t m2 = p * p, m3 = p * p * p, m4 = p * p * p * p;
    uint64_t h2 = 0, h1 = 0;
    for (uint64_t k = 1; k < p; ++k) {
        h2 = addmod(h2, invmod(mulmod(k, k, m2), m2), m2);
        h1 = addmod(h1, invmod(k, m3), m3);
    }
    uint64_t num = 1, den = 1;
    for (uint64_t k = 1; k < p; ++k) {
        num = mulmod(num, 2 * p - k, m4);
        den = mulmod(den, k, m4);
    }
    uint64_t c = mulmod(num, invmod(den, m4), m4);
    if (h2 == 0) bits |= 1;
    if (h1 == 0) bits |= 2;
    if (c == 1) bits |= 4;
    return bits;
}

/* ------------------------------------------------------------------ */
/* Level C: single-sum congruences with the accumulation of eqn 3.12   */
/* ------------------------------------------------------------------ */

/*
 * S(x,y) = sum_{xp < s < yp} s^-e  mod p   (eqn 2.3 with l = p-1-e, since
 * s^{p-1-e} = s^-e mod p), over the OPEN interval (xp, yp), x = xn/xd,
 * y = yn/yd.  If `alternating`, the sign (-1)^s is included (the sum
 * S~ of eqn 4.7).
 *
 * Evaluated with the polynomial trick of Sec. 3: prod (z + s^e) has
 * linear/constant coefficient ratio c1/c0 = sum s^-e, and eqn 3.12 builds
 * (c0, c1) one term at a time:  c1 <- c1 t + c0,  c0 <- c0 t,  t = s^e.
 * For the alternating sum, prod (z + (-1)^s s^e) is used instead, since
 * sum 1/((-1)^s s^e) = sum (-1)^s s^-e.
 */
uint64_t orc_interval_sum(uint64_t p, uint64_t xn, uint64_t xd, uint64_t yn,
                          uint64_t yd, unsigned e, int alternating) {
    /* first integer strictly above x p, last integer strictly below y p */
    u128 xp = (u128)xn * p, yp = (u128)yn * p;
    uint64_t lo = (uint64_t)(xp / xd) + 1;
    uint64_t hi = (uint64_t)((yp + yd - 1) / yd) - 1; /* ceil(yp) - 1 */
    uint64_t c0 = 1 % p, c1 = 0;
    for (uint64_t s = lo; s <= hi && s >= lo; ++s) {
        uint64_t t = powmod(s % p, e, p);
        if (alternating && (s & 1)) t = submod(0, t, p);
        c1 = addmod(mulmod(c1, t, p), c0, p);
        c0 = mulmod(c0, t, p);
    }
    if (c0 == 0) return UINT64_MAX;
    return mulmod(c1, invmod(c0, p), p);
}

/*
 * Stafford-Vandiver (Sec. 2, eqn 2.4) at k = (p-3)/2, i.e. eqn 3.2 (BB1):
 *   C_k(3,4,6) = (6^3 - 3^3 - 4^3 + 1)/6 = 21,   21 B_{p-3} = S(1/6, 1/4),
 * S = sum s^-3 (eqn 2.3 with l = p-4).  Valid for p >= 5, p != 7.
 */
uint64_t orc_bernoulli_sv(uint64_t p) {
    if (p < 5 || p == 7 || (p & 1) == 0) return UINT64_MAX;
    uint64_t S = orc_interval_sum(p, 1, 6, 1, 4, 3, 0);
    return mulmod(S, invmod(21 % p, p), p);
}

/*
 * Voronoi's form (Sec. 2, eqn 2.8) at k = (p-3)/2:
 *   C_k(2,3,4) = (4^3 - 2^3 - 3^3 + 1)/6 = 5,   5 B_{p-3} = S(1/4, 1/3).
 * Valid for p >= 7.
 */
uint64_t orc_bernoulli_v12(uint64_t p) {
    if (p < 7 || (p & 1) == 0) return UINT64_MAX;
    uint64_t S = orc_interval_sum(p, 1, 4, 1, 3, 3, 0);
    return mulmod(S, invmod(5, p), p);
}

/*
 * Glaisher's Euler congruence (Sec. 4, eqn 4.1) at k = 1 with the sign
 * factor (-1)^k (see the reading in the file header):
 *   -4 E_{p-3} = S_{p-3}(0, 1/4) = sum_{0<s<p/4} s^-2   (mod p),  p >= 5.
 */
uint64_t orc_euler_glaisher(uint64_t p) {
    if (p < 5 || (p & 1) == 0) return UINT64_MAX;
    uint64_t S = orc_interval_sum(p, 0, 1, 1, 4, 2, 0);
    return mulmod(submod(0, S, p), invmod(4, p), p);
}

/*
 * McIntosh's alternating congruence (Sec. 4, eqn 4.7) at k = 1:
 *   (-1)^1 4^0 (9 + 1) E_{p-3} = S~_{p-3}(0, 1/6)
 *   i.e.  -10 E_{p-3} = sum_{0<s<p/6} (-1)^s s^-2  (mod p),  p >= 7.
 */
uint64_t orc_euler_mcintosh(uint64_t p) {
    if (p < 7 || (p & 1) == 0) return UINT64_MAX;
    uint64_t S = orc_interval_sum(p, 0, 1, 1, 6, 2, 1);
    return mulmod(submod(0, S, p), invmod(10 % p, p), p);
}

/* Default large-p oracle pair: BB1/Stafford-Vandiver for B (Voronoi at p=7),
 * Glaisher eqn 4.1 for E.  p = 5 and 7 fall back to the definitions. */
uint64_t orc_bernoulli_pm3(uint64_t p) {
    if (p < 5 || (p & 1) == 0) return UINT64_MAX;
    if (p < 11) return orc_bernoulli_def(p - 3, p);
    return orc_bernoulli_sv(p);
}
uint64_t orc_euler_pm3(uint64_t p) {
    if (p < 5 || (p & 1) == 0) return UINT64_MAX;
    if (p < 11) return orc_euler_def(p - 3, p);
    return orc_euler_glaisher(p);
}

/* ------------------------------------------------------------------ */
/* threaded batch driver (one prime per task, plain pthreads)          */
/* ------------------------------------------------------------------ */
typedef struct {
    const uint64_t *primes;
    size_t n;
    uint64_t *out_b, *out_e;
    int method_b, method_e;
    size_t next;
    pthread_mutex_t mu;
} batch_job;

static uint64_t run_b(int method, uint64_t p) {
    switch (method) {
    case 0: return orc_bernoulli_pm3(p);
    case 1: return (p + 1 < 4) ? UINT64_MAX : orc_bernoulli_def(p - 3, p);
    case 2: return orc_bernoulli_h2(p);
    case 3: return orc_bernoulli_glaisher(p, 2);
    case 4: return orc_bernoulli_sv(p);
    case 5: return orc_bernoulli_v12(p);
    default: return UINT64_MAX;
    }
}
static uint64_t run_e(int method, uint64_t p) {
    switch (method) {
    case 0: return orc_euler_pm3(p);
    case 1: return (p < 4) ? UINT64_MAX : orc_euler_def(p - 3, p);
    case 6: return orc_euler_glaisher(p);
    case 7: return orc_euler_mcintosh(p);
    default: return UINT64_MAX;
    }
}

static void *batch_worker(void *arg) {
    batch_job *J = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        size_t i = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->n) break;
        uint64_t p = J->primes[i];
        if (J->out_b) J->out_b[i] = run_b(J->method_b, p);
        if (J->out_e) J->out_e[i] = run_e(J->method_e, p);
    }
    return NULL;
}

/*
 * Residues for a list of primes on `threads` host threads.  out_b / out_e
 * may be NULL.  method_b: 0 default, 1 definition, 2 harmonic, 3 Glaisher
 * binomial, 4 Stafford-Vandiver, 5 Voronoi.  method_e: 0 default,
 * 1 definition, 6 Glaisher eqn 4.1, 7 McIntosh eqn 4.7.
 */
int orc_residues(const uint64_t *primes, size_t n, uint64_t *out_b,
                 uint64_t *out_e, int method_b, int method_e, int threads) {
    if (threads < 1) threads = 1;
    batch_job J;
    J.primes = primes; J.n = n; J.out_b = out_b; J.out_e = out_e;
    J.method_b = method_b; J.method_e = method_e; J.next = 0;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    int started = 0;
    for (int i = 0; i < threads; ++i)
        if (pthread_create(&th[i], NULL, batch_worker, &J) == 0) ++started;
    if (started == 0) batch_worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    return 0;
}

/* ------------------------------------------------------------------ */
/* plain sieve of Eratosthenes on a window [lo, hi)                    */
/* ------------------------------------------------------------------ */
/*
 * Writes the primes of [lo, hi) in ascending order to out (at most cap of
 * them) and returns how many there are.  Base primes up to sqrt(hi) come
 * from a plain sieve; the window is a byte array (hi - lo must fit memory).
 */
uint64_t orc_sieve(uint64_t lo, uint64_t hi, uint64_t *out, uint64_t cap) {
    if (hi <= lo) return 0;
    uint64_t r = 1;
    while ((u128)(r + 1) * (r + 1) < hi) ++r;  /* r = ceil(sqrt(hi)) - ish */
    while ((u128)r * r >= hi && r > 1) --r;       /* r = max integer, r^2 < hi */
    uint8_t *small = (uint8_t *)calloc(r + 1, 1);    /* 1 = composite */
    uint64_t w = hi - lo;
    uint8_t *win = (uint8_t *)calloc(w, 1);
    if (!small || !win) { free(small); free(win); return UINT64_MAX; }
    for (uint64_t q = 2; q <= r; ++q) {
        if (small[q]) continue;
        for (uint64_t m = q * q; m <= r; m += q) small[m] = 1;
        /* cross off multiples of q in the window, starting at max(q^2, first multiple >= lo) */
        uint64_t start = (lo + q - 1) / q * q;
        if (start < q * q) start = q * q;
        for (uint64_t m = start; m < hi; m += q) win[m - lo] = 1;
    }
    uint64_t count = 0;
    for (uint64_t i = 0; i < w; ++i) {
        uint64_t v = lo + i;
        if (v < 2 || win[i]) continue;
        if (count < cap && out) out[count] = v;
        ++count;
    }
    free(small); free(win);
    return count;
}
