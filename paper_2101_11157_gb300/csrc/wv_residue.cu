// wv_residue.cu -- steps a2-a6: plan, term generation, accumulation, reduction
// and finalisation of B_{p-3} mod p and E_{p-3} mod p.
//
// Method (Sec. 3, "It remains to describe how to calculate these sums"; Sec. 5
// after eqn 5.6): every congruence row contributes coef * S(x, y) with
// S = sum_{xp<s<yp} s^-e (e = 3 for B_{p-3}, e = 2 for E_{p-3}).  S is the
// ratio c1/c0 of the two lowest coefficients of prod (z + s^e), built one
// term at a time by eqn 3.12 (c1 <- c1 t + c0, c0 <- c0 t, t = s^e); pieces
// of a product are merged with eqn 3.14.  One modular inverse per prime
// finishes the sum (Sec. 3, the CPU's last step in the paper's GPU method).
//
// GB300 design:
//  * Work unit = a warp tile: a contiguous range of s inside one (prime, row)
//    sum.  The planner splits every sum into at most `max_tiles` tiles of about
//    `tile_terms` terms.  A persistent kernel (grid = SMs x occupancy) lets
//    warps take tiles from an atomic counter, largest primes first.
//  * Inside a tile, 32 lanes x ILP chains each own a contiguous run of s.  Term
//    generation is by forward differences (Sec. 3, improvement 1): s^3 from
//    (s-1)^3 with three modular additions, s^2 with one; no multiplication.
//  * Accumulation: signed Montgomery arithmetic (see wv_arith.cuh).  For
//    p < 2^30 a term costs 7 integer multiplies (hi(c0 t), hi(c1 t), t p^-1,
//    c0 tq, c1 tq, hi(m0 p), hi(m1 p)); 64-bit words for 2^30 <= p < 2^37.
//  * The chains of a tile are merged with eqn 3.14 in registers and by warp
//    shuffles; one (c0, c1) pair per tile goes to global memory.  The finalise
//    kernel (one warp per prime and kind) merges the tiles of each sum, forms
//    sum_j coef_j c1_j / c0_j as one fraction, and inverts once (Fermat).
//
// Montgomery bookkeeping: the hot step multiplies by a plain t with REDC, so
// c0 and c1 drift by powers of R, but the ratio c1/c0 always equals S * R
// (true initially for (c0, c1) = (R, 0) and preserved by both eqn 3.12 steps
// and by eqn 3.14 under REDC).  The finaliser therefore divides by R once.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "wv_arith.cuh"
#include "wv_internal.h"
#include "wv_tables.h"

namespace wv {

constexpr int kAccThreads = 256;
constexpr int kMaxRowsPP = 66;  // B rows + E rows for one prime (30 + 33 for BB30 + EE33)
constexpr uint32_t kChunkPrimes = 16384;  // primes per internal launch sequence
constexpr uint64_t kGroupMinChain = 48;   // grouped path only for chains of >= 48 terms

struct Plan {
  uint32_t n;                   // primes in this chunk
  uint32_t rows_b, rows_e, rows_pp;
  uint32_t tile_terms, max_tiles;
  const uint64_t *primes;       // caller's primes (chunk base)
  uint64_t *out_b, *out_e;      // caller's outputs (chunk base), may be null
  PrimeCtx *ctx;                // per slot (M31 slots first, then M64)
  uint32_t *flag, *pos, *n31;   // flag: p-bucket per prime; n31: slots with p < 2^30
  uint32_t *bk;                 // 3 x 64 words: bucket counts, offsets, cursors
  uint64_t *seg_lo, *seg_cnt;   // per segment (slot * rows_pp + row)
  uint32_t *seg_tiles, *seg_first;
  uint32_t *total_tiles, *split_tile;
  uint32_t *counters;           // [0] M31 accumulation, [1] M64 accumulation
  ulonglong2 *partials;         // per tile (c0, c1), canonical
  // congruence rows: rows [0, rows_b) are B rows, [rows_b, rows_pp) E rows
  uint32_t xn[kMaxRowsPP], xd[kMaxRowsPP], yn[kMaxRowsPP], yd[kMaxRowsPP];
  int64_t coef[kMaxRowsPP];
  int64_t lhs_b, lhs_e;
};

// ------------------------------------------------------------------ planner
// Primes are ordered into slots by p-bucket floor(log2 p), ascending (a
// counting sort; order inside a bucket is arbitrary and does not affect any
// result).  Buckets 0..29 are the p < 2^30 slots; the accumulation kernels
// walk slots from the top, so the largest primes start first.
__device__ __forceinline__ uint32_t p_bucket(uint64_t p) {
  const bool valid = (p >= 11) && (p & 1) && (p < kPMax);
  return valid ? (uint32_t)(63 - __clzll((long long)p)) : 0u;  // special/invalid: no sums
}

__global__ void k_plan_prime(Plan P) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const uint32_t b = p_bucket(P.primes[i]);
  P.flag[i] = b;
  atomicAdd(&P.bk[b], 1u);
}

__global__ void k_plan_buckets(Plan P) {  // one warp: offsets of the 64 buckets
  const int lane = threadIdx.x;
  uint32_t c0 = P.bk[lane], c1 = P.bk[32 + lane];
  uint32_t x0 = c0, x1 = c1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
    if (lane >= o) { x0 += y0; x1 += y1; }
  }
  const uint32_t tot0 = __shfl_sync(0xffffffffu, x0, 31);
  P.bk[64 + lane] = x0 - c0;
  P.bk[96 + lane] = tot0 + x1 - c1;
  const uint32_t below30 = __shfl_sync(0xffffffffu, x0, 29);  // buckets 0..29
  if (lane == 0) *P.n31 = below30;
}

__global__ void k_plan_scatter(Plan P) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  uint64_t p = P.primes[i];
  const uint32_t b = P.flag[i];
  const uint32_t slot = P.bk[64 + b] + atomicAdd(&P.bk[128 + b], 1u);
  PrimeCtx c;
  bool valid = (p >= 5) && (p & 1) && (p < kPMax);
  if (valid && p >= 11) {
    c = make_ctx(p, i);
  } else {
    c.p = p; c.q = 0; c.one = 0; c.r2 = 0; c.orig = i;
    c.flags = 2u | ((p >= kM31Limit) ? 1u : 0u);  // no sums: special or invalid
  }
  P.ctx[slot] = c;
}

__global__ void k_plan_segments(Plan P) {
  uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.n * P.rows_pp) return;
  uint32_t slot = idx / P.rows_pp, j = idx - slot * P.rows_pp;
  const PrimeCtx c = P.ctx[slot];
  uint64_t lo = 0, cnt = 0;
  uint32_t tiles = 0;
  if (!(c.flags & 2u)) {
    const uint64_t p = c.p;
    // open interval (x p, y p): s = floor(xn p / xd) + 1 .. floor(yn p / yd)
    lo = (uint64_t)P.xn[j] * p / P.xd[j] + 1;
    uint64_t hi = (uint64_t)P.yn[j] * p / P.yd[j] + 1;
    cnt = hi > lo ? hi - lo : 0;
    if (cnt) {
      uint64_t t = (cnt + P.tile_terms - 1) / P.tile_terms;
      tiles = (uint32_t)(t < 1 ? 1 : (t > P.max_tiles ? P.max_tiles : t));
    }
  }
  P.seg_lo[idx] = lo;
  P.seg_cnt[idx] = cnt;
  P.seg_tiles[idx] = tiles;
}

__global__ void k_plan_split(Plan P) {
  uint32_t n31 = *P.n31;
  *P.split_tile = (n31 < P.n) ? P.seg_first[n31 * P.rows_pp] : *P.total_tiles;
  P.counters[0] = 0;
  P.counters[1] = 0;
}

// ------------------------------------------------------------------ tiles
// Warp-level merge of the per-lane pairs (eqn 3.14) through shuffles.
__device__ __forceinline__ void warp_merge(const Mont &M, int64_t &a0, int64_t &a1) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    int64_t b0 = __shfl_xor_sync(0xffffffffu, a0, o);
    int64_t b1 = __shfl_xor_sync(0xffffffffu, a1, o);
    M.combine(a0, a1, b0, b1);
  }
}

// p < 2^30: signed 32-bit Montgomery, R = 2^32.  AR selects the product
// formulation: 1 = hi(c t) and lo(c tq) with tq = t p^-1 shared by c0 and c1;
// 2 = the full 64-bit product c t (one wide multiply) and m = lo(c t) p^-1.
template <int ILP, bool CUBES, int AR>
__device__ __forceinline__ void tile_m31(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                         int64_t &r0, int64_t &r1) {
  const int lane = threadIdx.x & 31;
  const int32_t p = (int32_t)ctx.p;
  const uint32_t up = (uint32_t)ctx.p;
  const uint32_t q = (uint32_t)ctx.q;
  const uint64_t nch = 32 * ILP;
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  int32_t c0[ILP], c1[ILP], t[ILP], d1[ILP], d2[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = k * 32 + lane;
    const uint64_t s = start + ch * len + (ch < rem ? ch : rem);
    const uint64_t s2 = (s * s) % ctx.p;  // s < 2^30: exact in 64 bits
    if (CUBES) {
      t[k] = (int32_t)((s2 * s) % ctx.p);              // s^3
      d1[k] = (int32_t)((3 * s2 + 3 * s + 1) % ctx.p); // (s+1)^3 - s^3
      d2[k] = (int32_t)((6 * s + 6) % ctx.p);          // second difference
    } else {
      t[k] = (int32_t)s2;                              // s^2
      d1[k] = (int32_t)(2 * s + 1);                    // (s+1)^2 - s^2 <= p (s < p/2)
      d2[k] = 0;
    }
    c0[k] = (int32_t)ctx.one;
    c1[k] = 0;
  }
  // z: a runtime zero (the context's upper flag bits are never set) that the
  // compiler cannot fold.  Written into otherwise two-input additions it makes
  // them genuine three-input adds, which only the integer ALU executes, so
  // they stay off the multiply pipe the products saturate (AR >= 3).
  const int32_t z = (int32_t)(ctx.flags >> 16);
  const int32_t np = -p;
  auto step = [&](int k, int32_t zi) {
    // eqn 3.12 with REDC against the plain term t
    if (AR == 1) {
      const uint32_t tq = (uint32_t)t[k] * q;
      const int32_t m0 = (int32_t)((uint32_t)c0[k] * tq);
      const int32_t m1 = (int32_t)((uint32_t)c1[k] * tq);
      const int32_t h0 = __mulhi(c0[k], t[k]);
      const int32_t h1 = __mulhi(c1[k], t[k]);
      const int32_t n1 = h1 - __mulhi(m1, p) + c0[k];
      c0[k] = h0 - __mulhi(m0, p);
      c1[k] = n1;
    } else if (AR >= 6) {
      // REDC folded into a wide multiply-add: d = w - m p is an exact
      // multiple of 2^32 whose high word is the reduced value, and c0 rides
      // in the high word of c1's product, so no separate add is needed.
      const int64_t w0 = mul_wide(c0[k], t[k]);
      const int64_t w1 = mad_wide(c1[k], t[k], hi_word(c0[k]));
      const int32_t m0 = (int32_t)((uint32_t)lo32(w0) * q);
      const int32_t m1 = (int32_t)((uint32_t)lo32(w1) * q);
      c0[k] = hi32(mad_wide(m0, np, w0));
      c1[k] = hi32(mad_wide(m1, np, w1));
    } else {
      const int64_t w0 = (int64_t)c0[k] * (int64_t)t[k];
      const int64_t w1 = (int64_t)c1[k] * (int64_t)t[k];
      const int32_t m0 = (int32_t)((uint32_t)w0 * q);
      const int32_t m1 = (int32_t)((uint32_t)w1 * q);
      const int32_t n1 = (int32_t)(w1 >> 32) - __mulhi(m1, p) + c0[k];
      if (AR >= 3) c0[k] = (int32_t)(w0 >> 32) - __mulhi(m0, p) + zi;
      else c0[k] = (int32_t)(w0 >> 32) - __mulhi(m0, p);
      c1[k] = n1;
    }
    // forward differences, each a modular add as min(x, x - p) on unsigned words
    const uint32_t uz = (uint32_t)(AR >= 3 && AR < 6 ? z : 0);
    const uint32_t uzi = (uint32_t)(AR >= 4 && AR < 6 ? zi : 0);
    uint32_t x = (uint32_t)t[k] + (uint32_t)d1[k] + uz;
    uint32_t y = (uint32_t)t[k] + (uint32_t)d1[k] - up;
    t[k] = (int32_t)min(x, y);
    if (CUBES) {
      x = (uint32_t)d1[k] + (uint32_t)d2[k] + uz;
      y = (uint32_t)d1[k] + (uint32_t)d2[k] - up;
      d1[k] = (int32_t)min(x, y);
      x = (uint32_t)d2[k] + 6u + uzi;
      y = (uint32_t)d2[k] + (6u - up) + uzi;
      d2[k] = (int32_t)min(x, y);
    } else {
      d1[k] = (int32_t)((uint32_t)d1[k] + 2u + uzi);
    }
  };
#pragma unroll 2
  for (uint64_t it = 0; it < len; ++it) {
    // a per-iteration zero (chains never reach 2^63 terms)
    const int32_t zi = (AR >= 4 && AR < 6) ? (int32_t)(it >> 63) : z;
#pragma unroll
    for (int k = 0; k < ILP; ++k) step(k, zi);
  }
#pragma unroll
  for (int k = 0; k < ILP; ++k)
    if ((uint32_t)(k * 32 + lane) < rem) step(k, z);

  const Mont M(ctx);
  int64_t a0 = m31_canon(c0[0], p), a1 = m31_canon(c1[0], p);
#pragma unroll
  for (int k = 1; k < ILP; ++k) M.combine(a0, a1, m31_canon(c0[k], p), m31_canon(c1[k], p));
  warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// ---- grouped accumulation (p < 2^30) ------------------------------------
// eqn 3.14 applied to a GROUP of K consecutive terms: the group's factor
// prod_{i<K} (z + (s+i)^e) = G0(s) + G1(s) z + O(z^2) with
//   G0(s) = prod_i (s+i)^e,   G1(s) = sum_i prod_{j!=i} (s+j)^e,
// polynomials in s of degree K e and (K-1) e.  Both are stepped s -> s+K by
// forward differences (additions only), and each group costs three products:
//   c0 <- c0 G0,   c1 <- c1 G0 + c0 G1.
// G1 is kept in Montgomery form so that, as in the single-term step, the
// ratio c1/c0 accumulates R * sum t^-1 (see the bookkeeping note above).

// G0(x) (plain) and G1(x) R (Montgomery) for the group x, x+1, ..., x+K-1.
template <int K, int EX>
__device__ __forceinline__ void group_poly(const Mont &M, uint64_t x, int64_t &g0, int64_t &g1m) {
  int64_t tm[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    uint64_t v = x + i;
    if (v >= (uint64_t)M.p) v -= (uint64_t)M.p;
    const int64_t b = M.to_mont((int64_t)v);
    int64_t t = M.mul(b, b);
    if (EX == 3) t = M.mul(t, b);
    tm[i] = t;  // (x+i)^e in Montgomery form
  }
  int64_t all = M.one, g1 = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    int64_t others = M.one;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j != i) others = M.mul(others, tm[j]);
    g1 = M.add(g1, others);
    all = M.mul(all, tm[i]);
  }
  g0 = M.from_mont(all);
  g1m = g1;
}

template <int ILP, bool CUBES, int AR>
__device__ __forceinline__ void tile_m31_grouped(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                                 int64_t &r0, int64_t &r1) {
  constexpr int K = CUBES ? 2 : 3;     // terms per group
  constexpr int EX = CUBES ? 3 : 2;    // t = s^EX
  constexpr int DA = K * EX;           // degree of G0
  constexpr int DB = (K - 1) * EX;     // degree of G1
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  const int32_t p = (int32_t)ctx.p;
  const uint32_t up = (uint32_t)ctx.p;
  const uint32_t q = (uint32_t)ctx.q;
  const uint32_t uz = (AR >= 7) ? 0u : (ctx.flags >> 16);  // runtime zero (AR 5: three-input adds)
  const int32_t np = -p;
  const uint64_t nch = 32 * ILP;
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  const uint64_t G = len / K;  // groups per chain, the same for every lane
  int32_t c0[ILP], c1[ILP], ga[ILP][DA + 1], gb[ILP][DB + 1];
  uint64_t s_tail[ILP];
  uint32_t n_tail[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = k * 32 + lane;
    const uint64_t s = start + ch * len + (ch < rem ? ch : rem);
    const uint64_t L = len + (ch < rem ? 1 : 0);
    s_tail[k] = s + G * K;
    n_tail[k] = (uint32_t)(L - G * K);
    // difference tables of G0 and G1 at s, s+K, s+2K, ...
    int64_t va[DA + 1], vb[DB + 1];
#pragma unroll
    for (int i = 0; i <= DA; ++i) {
      int64_t a, b;
      group_poly<K, EX>(M, s + (uint64_t)i * K, a, b);
      va[i] = a;
      if (i <= DB) vb[i] = b;
    }
#pragma unroll
    for (int j = 1; j <= DA; ++j)
#pragma unroll
      for (int i = DA; i >= j; --i) va[i] = M.sub(va[i], va[i - 1]);
#pragma unroll
    for (int j = 1; j <= DB; ++j)
#pragma unroll
      for (int i = DB; i >= j; --i) vb[i] = M.sub(vb[i], vb[i - 1]);
#pragma unroll
    for (int i = 0; i <= DA; ++i) ga[k][i] = (int32_t)va[i];
#pragma unroll
    for (int i = 0; i <= DB; ++i) gb[k][i] = (int32_t)vb[i];
    c0[k] = (int32_t)ctx.one;
    c1[k] = 0;
  }
  auto modadd = [&](int32_t &a, int32_t b) {
    const uint32_t x = (uint32_t)a + (uint32_t)b + uz;
    const uint32_t y = (uint32_t)a + (uint32_t)b - up;
    a = (int32_t)min(x, y);
  };
#pragma unroll 1
  for (uint64_t g = 0; g < G; ++g) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
      const int32_t A = ga[k][0], B = gb[k][0];
      if (AR >= 7) {
        // one REDC for c1 G0 + c0 G1 R, folded into wide multiply-adds
        const int64_t w0 = mul_wide(c0[k], A);
        const int64_t w1 = mad_wide(c0[k], B, mul_wide(c1[k], A));
        const int32_t m0 = (int32_t)((uint32_t)lo32(w0) * q);
        const int32_t m1 = (int32_t)((uint32_t)lo32(w1) * q);
        c0[k] = hi32(mad_wide(m0, np, w0));
        c1[k] = hi32(mad_wide(m1, np, w1));
      } else {
        const int64_t w0 = (int64_t)c0[k] * (int64_t)A;
        const int64_t w1 = (int64_t)c1[k] * (int64_t)A;
        const int64_t w2 = (int64_t)c0[k] * (int64_t)B;
        const int32_t m0 = (int32_t)((uint32_t)w0 * q);
        const int32_t m1 = (int32_t)((uint32_t)w1 * q);
        const int32_t m2 = (int32_t)((uint32_t)w2 * q);
        const int32_t n1 = ((int32_t)(w1 >> 32) - __mulhi(m1, p)) + ((int32_t)(w2 >> 32) - __mulhi(m2, p));
        c0[k] = (int32_t)(w0 >> 32) - __mulhi(m0, p) + (int32_t)uz;
        c1[k] = n1;
      }
      // step both difference tables by one group (low order first)
#pragma unroll
      for (int j = 0; j < DA; ++j) modadd(ga[k][j], ga[k][j + 1]);
#pragma unroll
      for (int j = 0; j < DB; ++j) modadd(gb[k][j], gb[k][j + 1]);
    }
  }
  // the last (at most K) terms of each chain one at a time (eqn 3.12)
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if ((uint32_t)i < n_tail[k]) {
        const int64_t b = M.to_mont((int64_t)(s_tail[k] + i));
        int64_t tm = M.mul(b, b);
        if (EX == 3) tm = M.mul(tm, b);
        const int32_t t = (int32_t)M.from_mont(tm);
        const int64_t w0 = (int64_t)c0[k] * (int64_t)t;
        const int64_t w1 = (int64_t)c1[k] * (int64_t)t;
        const int32_t m0 = (int32_t)((uint32_t)w0 * q);
        const int32_t m1 = (int32_t)((uint32_t)w1 * q);
        const int32_t n1 = (int32_t)(w1 >> 32) - __mulhi(m1, p) + c0[k];
        c0[k] = (int32_t)(w0 >> 32) - __mulhi(m0, p);
        c1[k] = n1;
      }
    }
  }
  int64_t a0 = m31_canon(c0[0], p), a1 = m31_canon(c1[0], p);
#pragma unroll
  for (int k = 1; k < ILP; ++k) M.combine(a0, a1, m31_canon(c0[k], p), m31_canon(c1[k], p));
  warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// 2^30 <= p < 2^37: signed 64-bit Montgomery, R = 2^64.
template <int ILP, bool CUBES>
__device__ __forceinline__ void tile_m64(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                         int64_t &r0, int64_t &r1) {
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  const int64_t p = (int64_t)ctx.p;
  const uint64_t up = ctx.p;
  const uint64_t q = ctx.q;
  const uint64_t nch = 32 * ILP;
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  int64_t c0[ILP], c1[ILP], t[ILP], d1[ILP], d2[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = k * 32 + lane;
    const uint64_t s = start + ch * len + (ch < rem ? ch : rem);
    const int64_t s2 = M.mulmod((int64_t)s, (int64_t)s);
    if (CUBES) {
      t[k] = M.mulmod(s2, (int64_t)s);
      d1[k] = (int64_t)((3 * (uint64_t)s2 + 3 * s + 1) % up);
      d2[k] = (int64_t)((6 * s + 6) % up);
    } else {
      t[k] = s2;
      d1[k] = (int64_t)(2 * s + 1);
      d2[k] = 0;
    }
    c0[k] = (int64_t)ctx.one;
    c1[k] = 0;
  }
  auto step = [&](int k) {
    const uint64_t tq = (uint64_t)t[k] * q;
    const int64_t m0 = (int64_t)((uint64_t)c0[k] * tq);
    const int64_t m1 = (int64_t)((uint64_t)c1[k] * tq);
    const int64_t h0 = __mul64hi(c0[k], t[k]);
    const int64_t h1 = __mul64hi(c1[k], t[k]);
    const int64_t n1 = h1 - __mul64hi(m1, p) + c0[k];
    c0[k] = h0 - __mul64hi(m0, p);
    c1[k] = n1;
    uint64_t x = (uint64_t)t[k] + (uint64_t)d1[k];
    t[k] = (int64_t)min(x, x - up);
    if (CUBES) {
      x = (uint64_t)d1[k] + (uint64_t)d2[k];
      d1[k] = (int64_t)min(x, x - up);
      x = (uint64_t)d2[k] + 6u;
      d2[k] = (int64_t)min(x, x - up);
    } else {
      d1[k] += 2;
    }
  };
#pragma unroll 1
  for (uint64_t it = 0; it < len; ++it) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) step(k);
  }
#pragma unroll
  for (int k = 0; k < ILP; ++k)
    if ((uint32_t)(k * 32 + lane) < rem) step(k);

  int64_t a0 = m64_canon(c0[0], p), a1 = m64_canon(c1[0], p);
#pragma unroll
  for (int k = 1; k < ILP; ++k) M.combine(a0, a1, m64_canon(c0[k], p), m64_canon(c1[k], p));
  warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// ---- grouped accumulation for 2^30 <= p < 2^37 ------------------------------
// Montgomery with R = 2^64 done as two 32-bit rounds on unsigned words:
// p = p0 + p1 2^32 (p1 < 32), q = -p^-1 mod 2^32.  A product T = c g is held
// as a low word T0 and a 64-bit rest TY (T = T0 + TY 2^32); each round adds
// m p with m = (low word) q, which clears the low word exactly.  For
// c < 2^38 and g < 2^53 every intermediate fits its word and the result is
// below p + 2^24 (one conditional subtraction makes it canonical).
//
// The group polynomials of the grouped scheme above are stepped with plain
// 64-bit additions and no reduction; every kM64Block groups the tables are
// brought back below 10 p by an approximate Barrett step (quotient from the
// high word times floor(2^62 / p)).  Starting below 10 p, a degree-6 table
// stays below 10 p C(8+6, 6) < 2^52 over a block, inside the product bound.
constexpr uint32_t kM64Block = 8;

struct M64K {
  uint32_t p0, p1, q, mhi;  // mhi = floor(2^62 / p)
  uint64_t p;
};

__device__ __forceinline__ uint64_t umul_wide(uint32_t a, uint32_t b) {
  uint64_t d;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint64_t umad_wide(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint32_t ulo(uint64_t v) {
  uint32_t lo;
  asm("{\n\t.reg .b32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=r"(lo) : "l"(v));
  return lo;
}
__device__ __forceinline__ uint32_t uhi(uint64_t v) {
  uint32_t hi;
  asm("{\n\t.reg .b32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=r"(hi) : "l"(v));
  return hi;
}
__device__ __forceinline__ uint64_t upack(uint32_t lo, uint32_t hi) {
  uint64_t v;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "r"(lo), "r"(hi));
  return v;
}

// (T0 + TY 2^32) 2^-64 mod p, result < p + 2^24
__device__ __forceinline__ uint64_t m64_redc2(uint32_t T0, uint64_t TY, const M64K &K) {
  const uint32_t m0 = T0 * K.q;
  const uint64_t A = umad_wide(m0, K.p0, (uint64_t)T0);       // low word is 0
  const uint64_t U = umad_wide(m0, K.p1, TY) + uhi(A);        // (T + m0 p) / 2^32
  const uint32_t m1 = ulo(U) * K.q;
  const uint64_t B = umad_wide(m1, K.p0, (uint64_t)ulo(U));   // low word is 0
  return umad_wide(m1, K.p1, (uint64_t)uhi(U)) + uhi(B);      // (U + m1 p) / 2^32
}
// T = c g as (T0, TY); c < 2^38, g < 2^53
__device__ __forceinline__ void m64_prod(uint64_t c, uint64_t g, uint32_t &T0, uint64_t &TY) {
  const uint32_t c0 = ulo(c), c1 = uhi(c), g0 = ulo(g), g1 = uhi(g);
  const uint64_t X = umul_wide(c0, g0);
  T0 = ulo(X);
  uint64_t Y = umad_wide(c0, g1, (uint64_t)uhi(X));
  Y = umad_wide(c1, g0, Y);
  TY = upack(ulo(Y), uhi(Y) + c1 * g1);
}
// T = ca ga + cb gb as (T0, TY)
__device__ __forceinline__ void m64_prod2(uint64_t ca, uint64_t ga, uint64_t cb, uint64_t gb,
                                          uint32_t &T0, uint64_t &TY) {
  const uint32_t a0 = ulo(ca), a1 = uhi(ca), x0 = ulo(ga), x1 = uhi(ga);
  const uint32_t b0 = ulo(cb), b1 = uhi(cb), y0 = ulo(gb), y1 = uhi(gb);
  const uint64_t Xa = umul_wide(a0, x0);
  const uint64_t Xb = umad_wide(b0, y0, (uint64_t)ulo(Xa));
  T0 = ulo(Xb);
  uint64_t Y = umad_wide(a0, x1, (uint64_t)uhi(Xa));
  Y = umad_wide(a1, x0, Y);
  Y = umad_wide(b0, y1, Y);
  Y = umad_wide(b1, y0, Y) + uhi(Xb);
  TY = upack(ulo(Y), uhi(Y) + a1 * x1 + b1 * y1);
}
// v < 2^64  ->  v' = v (mod p) with v' < 10 p
__device__ __forceinline__ uint64_t m64_shrink(uint64_t v, const M64K &K) {
  const uint64_t qq = umul_wide(uhi(v), K.mhi) >> 30;  // <= floor(v / p), short by < 10
  const uint32_t q0 = ulo(qq), q1 = uhi(qq);
  const uint64_t qp = umul_wide(q0, K.p0) + ((uint64_t)(q0 * K.p1 + q1 * K.p0) << 32);
  return v - qp;
}

template <int ILP, bool CUBES>
__device__ __forceinline__ void tile_m64_grouped(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                                 int64_t &r0, int64_t &r1) {
  constexpr int K = CUBES ? 2 : 3;
  constexpr int EX = CUBES ? 3 : 2;
  constexpr int DA = K * EX;
  constexpr int DB = (K - 1) * EX;
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  M64K KK;
  KK.p = ctx.p;
  KK.p0 = (uint32_t)ctx.p;
  KK.p1 = (uint32_t)(ctx.p >> 32);
  KK.q = 0u - (uint32_t)ctx.q;  // -p^-1 mod 2^32
  KK.mhi = (uint32_t)((1ull << 62) / ctx.p);
  const uint64_t nch = 32 * ILP;
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  const uint64_t G = len / K;
  uint64_t c0[ILP], c1[ILP], ga[ILP][DA + 1], gb[ILP][DB + 1];
  uint64_t s_tail[ILP];
  uint32_t n_tail[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = k * 32 + lane;
    const uint64_t s = start + ch * len + (ch < rem ? ch : rem);
    const uint64_t L = len + (ch < rem ? 1 : 0);
    s_tail[k] = s + G * K;
    n_tail[k] = (uint32_t)(L - G * K);
    int64_t va[DA + 1], vb[DB + 1];
#pragma unroll
    for (int i = 0; i <= DA; ++i) {
      int64_t a, b;
      group_poly<K, EX>(M, s + (uint64_t)i * K, a, b);
      va[i] = a;
      if (i <= DB) vb[i] = b;
    }
#pragma unroll
    for (int j = 1; j <= DA; ++j)
#pragma unroll
      for (int i = DA; i >= j; --i) va[i] = M.sub(va[i], va[i - 1]);
#pragma unroll
    for (int j = 1; j <= DB; ++j)
#pragma unroll
      for (int i = DB; i >= j; --i) vb[i] = M.sub(vb[i], vb[i - 1]);
#pragma unroll
    for (int i = 0; i <= DA; ++i) ga[k][i] = (uint64_t)va[i];
#pragma unroll
    for (int i = 0; i <= DB; ++i) gb[k][i] = (uint64_t)vb[i];
    c0[k] = ctx.one;
    c1[k] = 0;
  }
  for (uint64_t g = 0; g < G;) {
    const uint32_t nb = (G - g < kM64Block) ? (uint32_t)(G - g) : kM64Block;
#pragma unroll 1
    for (uint32_t r = 0; r < nb; ++r) {
#pragma unroll
      for (int k = 0; k < ILP; ++k) {
        uint32_t T0;
        uint64_t TY;
        m64_prod(c0[k], ga[k][0], T0, TY);
        const uint64_t n0 = m64_redc2(T0, TY, KK);
        m64_prod2(c1[k], ga[k][0], c0[k], gb[k][0], T0, TY);
        c1[k] = m64_redc2(T0, TY, KK);
        c0[k] = n0;
#pragma unroll
        for (int j = 0; j < DA; ++j) ga[k][j] += ga[k][j + 1];
#pragma unroll
        for (int j = 0; j < DB; ++j) gb[k][j] += gb[k][j + 1];
      }
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
#pragma unroll
      for (int j = 0; j < DA; ++j) ga[k][j] = m64_shrink(ga[k][j], KK);
#pragma unroll
      for (int j = 0; j < DB; ++j) gb[k][j] = m64_shrink(gb[k][j], KK);
    }
    g += nb;
  }
  // canonical accumulators, then the last (at most K) terms one at a time
  int64_t a0 = 0, a1 = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    int64_t x0 = (int64_t)(c0[k] >= ctx.p ? c0[k] - ctx.p : c0[k]);
    int64_t x1 = (int64_t)(c1[k] >= ctx.p ? c1[k] - ctx.p : c1[k]);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if ((uint32_t)i < n_tail[k]) {
        const int64_t b = M.to_mont((int64_t)(s_tail[k] + i));
        int64_t tm = M.mul(b, b);
        if (EX == 3) tm = M.mul(tm, b);
        const int64_t t = M.from_mont(tm);
        x1 = M.add(M.mul(x1, t), x0);  // REDC(c1 t) + c0, as in eqn 3.12's single step
        x0 = M.mul(x0, t);
      }
    }
    if (k == 0) {
      a0 = x0;
      a1 = x1;
    } else {
      M.combine(a0, a1, x0, x1);
    }
  }
  warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// ------------------------------------------------------------------ accumulate
// One warp tile g of plan P: find its (prime, row) segment, sum its range of
// terms, merge the lanes, and store the tile's (c0, c1) pair.
template <bool WIDE, int ILP, int AR>
__device__ __forceinline__ void process_tile(const Plan &P, uint32_t g) {
  const int lane = threadIdx.x & 31;
  const uint32_t nsegs = P.n * P.rows_pp;
  // segment owning tile g: the last s with seg_first[s] <= g
  uint32_t lo = 0, hi = nsegs;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&P.seg_first[mid]) <= g) lo = mid; else hi = mid;
  }
  const uint32_t s = lo;
  const uint32_t slot = s / P.rows_pp, j = s - slot * P.rows_pp;
  const PrimeCtx ctx = P.ctx[slot];
  const uint32_t k = g - P.seg_first[s], T = P.seg_tiles[s];
  const uint64_t cnt = P.seg_cnt[s];
  const uint64_t b0 = cnt * k / T, b1 = cnt * (k + 1) / T;
  const uint64_t start = P.seg_lo[s] + b0, n = b1 - b0;
  int64_t r0, r1;
  // single-term form used beside the grouped one
  constexpr int AS = (AR == 5 || AR == 8 || AR == 9) ? 4 : AR;
  const bool grp_ok = n >= 32ull * ILP * kGroupMinChain;
  if (!WIDE && AR == 5 && grp_ok) {
    if (j < P.rows_b) tile_m31_grouped<ILP, true, 5>(ctx, start, n, r0, r1);
    else tile_m31_grouped<ILP, false, 5>(ctx, start, n, r0, r1);
  } else if (!WIDE && AR >= 7 && grp_ok && j >= P.rows_b) {
    tile_m31_grouped<ILP, false, 7>(ctx, start, n, r0, r1);
  } else if (!WIDE && AR == 9 && grp_ok) {
    tile_m31_grouped<ILP, true, 7>(ctx, start, n, r0, r1);
  } else if (!WIDE) {
    if (j < P.rows_b) tile_m31<ILP, true, AS>(ctx, start, n, r0, r1);
    else tile_m31<ILP, false, AS>(ctx, start, n, r0, r1);
  } else if (AR >= 9 && grp_ok) {
    if (j < P.rows_b) tile_m64_grouped<ILP, true>(ctx, start, n, r0, r1);
    else tile_m64_grouped<ILP, false>(ctx, start, n, r0, r1);
  } else {
    if (j < P.rows_b) tile_m64<ILP, true>(ctx, start, n, r0, r1);
    else tile_m64<ILP, false>(ctx, start, n, r0, r1);
  }
  if (lane == 0) P.partials[g] = make_ulonglong2((unsigned long long)r0, (unsigned long long)r1);
}

template <bool WIDE, int ILP, int AR>
__global__ void __launch_bounds__(kAccThreads) k_accumulate(Plan P) {
  const int lane = threadIdx.x & 31;
  const uint32_t total = *P.total_tiles, split = *P.split_tile;
  const uint32_t t_begin = WIDE ? split : 0u, t_end = WIDE ? total : split;
  const uint32_t ntiles = t_end - t_begin;
  uint32_t *counter = P.counters + (WIDE ? 1 : 0);
  for (;;) {
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(counter, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= ntiles) break;
    process_tile<WIDE, ILP, AR>(P, t_end - 1 - g);  // largest primes first
  }
}

// Epoch form: tiles of several plans (one per request of a serving loop),
// given as items {plan, first tile, count, prefix}; the items' tiles are
// taken from one counter, each item from its top tile down.
template <bool WIDE, int ILP, int AR>
__global__ void __launch_bounds__(kAccThreads)
    k_epoch(const EpochItem *items, uint32_t n_items, uint32_t total, const Plan *plans,
            uint32_t *counter) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(counter, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= total) break;
    uint32_t lo = 0, hi = n_items;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&items[mid].prefix) <= g) lo = mid; else hi = mid;
    }
    const EpochItem it = items[lo];
    process_tile<WIDE, ILP, AR>(plans[it.plan], it.first + it.count - 1 - (g - it.prefix));
  }
}

// Epoch form with both arithmetic paths in one launch: items with bit 31 of
// `plan` set are 64-bit-path tiles.  One launch (and one tail) per epoch.
template <int ILP>
__global__ void __launch_bounds__(kAccThreads)
    k_epoch_mixed(const EpochItem *items, uint32_t n_items, uint32_t total, const Plan *plans,
                  uint32_t *counter) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(counter, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= total) break;
    uint32_t lo = 0, hi = n_items;
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&items[mid].prefix) <= g) lo = mid; else hi = mid;
    }
    const EpochItem it = items[lo];
    const uint32_t tile = it.first + it.count - 1 - (g - it.prefix);
    if (it.plan >> 31) process_tile<true, ILP, 9>(plans[it.plan & 0x7fffffffu], tile);
    else process_tile<false, ILP, 9>(plans[it.plan], tile);
  }
}

// ------------------------------------------------------------------ finalize
__device__ __forceinline__ int64_t smod64(int64_t c, int64_t p) {
  int64_t r = c % p;
  return r < 0 ? r + p : r;
}

// B_{p-3}, E_{p-3} mod p for p = 5, 7 (where some LHS constants vanish):
// B_2 = 1/6 = 1 mod 5, E_2 = 1;  B_4 = -1/30 = 3 mod 7, E_4 = 5.
__device__ __forceinline__ uint64_t special_value(uint64_t p, bool isB) {
  if (p == 5) return 1;
  if (p == 7) return isB ? 3 : 5;
  return WV_RESIDUE_INVALID;
}

__global__ void k_finalize(Plan P) {
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nk = (P.rows_b ? 1u : 0u) + (P.rows_e ? 1u : 0u);
  if (gw >= P.n * nk) return;
  const uint32_t slot = gw / nk, kk = gw - slot * nk;
  const bool isB = (P.rows_b != 0) && kk == 0;
  uint64_t *out = isB ? P.out_b : P.out_e;
  if (!out) return;
  const PrimeCtx ctx = P.ctx[slot];
  if (ctx.flags & 2u) {
    if (lane == 0) out[ctx.orig] = special_value(ctx.p, isB);
    return;
  }
  const Mont M(ctx);
  const int64_t p = (int64_t)ctx.p;
  const uint32_t nrows = isB ? P.rows_b : P.rows_e;
  const uint32_t r0 = isB ? 0u : P.rows_b;
  const uint32_t seg0 = slot * P.rows_pp + r0;
  int64_t N = 0, D = M.one;  // running fraction N / D = sum coef_j c1_j / c0_j
  for (uint32_t j = lane; j < nrows; j += 32) {
    const uint32_t s = seg0 + j;
    int64_t C0 = M.one, C1 = 0;
    const uint32_t f = P.seg_first[s], T = P.seg_tiles[s];
    for (uint32_t g = f; g < f + T; ++g) {
      const ulonglong2 v = P.partials[g];
      M.combine(C0, C1, (int64_t)v.x, (int64_t)v.y);
    }
    const int64_t aM = M.to_mont(smod64(P.coef[r0 + j], p));
    const int64_t X = M.mul(aM, C1);  // coef * C1 at C1's scale
    N = M.add(M.mul(N, C0), M.mul(X, D));
    D = M.mul(D, C0);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const int64_t N2 = __shfl_xor_sync(0xffffffffu, N, o);
    const int64_t D2 = __shfl_xor_sync(0xffffffffu, D, o);
    N = M.add(M.mul(N, D2), M.mul(N2, D));
    D = M.mul(D, D2);
  }
  if (lane == 0) {
    const int64_t L = smod64(isB ? P.lhs_b : P.lhs_e, p);
    if (L == 0 || D == 0) {
      out[ctx.orig] = WV_RESIDUE_INVALID;
      return;
    }
    // residue = (N/D) R^-1 / L = N / (D L R)
    const int64_t DLR = M.mul(D, M.to_mont(M.to_mont(L)));  // D * L R^2 * R^-1
    const int64_t inv = M.pow(M.to_mont(DLR), (uint64_t)(p - 2));  // (DLR)^-1 R
    out[ctx.orig] = (uint64_t)M.mul(N, inv);                 // N (DLR)^-1
  }
}

// ------------------------------------------------------------------ host
template <bool WIDE>
static wv_status launch_accumulate(const Plan &P, const ResidueConfig &cfg, int sms, cudaStream_t s) {
  const char *name = WIDE ? "accumulate_m64" : "accumulate_m31";
  void (*kern)(Plan) = nullptr;
  const int ar = WIDE ? (cfg.arith >= 9 ? 9 : 1) : cfg.arith;
#define WV_PICK(I)                                                          \
  (ar == 1 ? k_accumulate<WIDE, I, 1> : ar == 2 ? k_accumulate<WIDE, I, 2> \
   : ar == 3 ? k_accumulate<WIDE, I, 3> : ar == 4 ? k_accumulate<WIDE, I, 4> \
   : ar == 5 ? k_accumulate<WIDE, I, 5> : ar == 6 ? k_accumulate<WIDE, I, 6>  \
   : ar == 7 ? k_accumulate<WIDE, I, 7> : ar == 8 ? k_accumulate<WIDE, I, 8>  \
   : k_accumulate<WIDE, I, 9>)
  switch (cfg.ilp) {
    case 1: kern = WV_PICK(1); break;
    case 2: kern = WV_PICK(2); break;
    default: kern = WV_PICK(4); break;
  }
#undef WV_PICK
  int occ = cfg.blocks_per_sm;
  if (occ <= 0) {
    WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAccThreads, 0));
    if (occ < 1) occ = 1;
  }
  WV_LAUNCH(name, kern, (unsigned)(sms * occ), kAccThreads, 0, s, P);
  return WV_OK;
}

wv_status residues_device(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                          uint64_t *d_out_e, const ResidueConfig &cfg, cudaStream_t s) {
  if (n == 0) return WV_OK;
  if (!d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));
  Plan P;
  memset(&P, 0, sizeof P);
  const bool do_b = cfg.cong_b >= 0 && d_out_b;
  const bool do_e = cfg.cong_e >= 0 && d_out_e;
  if (!do_b && !do_e) return WV_OK;
  uint32_t r = 0;
  if (do_b) {
    const WvCongruence &c = kWvCongruences[cfg.cong_b];
    for (int j = 0; j < c.nrows; ++j, ++r) {
      const WvRow &w = kWvRows[c.row_offset + j];
      P.xn[r] = w.xn; P.xd[r] = w.xd; P.yn[r] = w.yn; P.yd[r] = w.yd; P.coef[r] = w.coef;
    }
    P.rows_b = c.nrows;
    P.lhs_b = c.lhs;
  }
  if (do_e) {
    const WvCongruence &c = kWvCongruences[cfg.cong_e];
    for (int j = 0; j < c.nrows; ++j, ++r) {
      const WvRow &w = kWvRows[c.row_offset + j];
      P.xn[r] = w.xn; P.xd[r] = w.xd; P.yn[r] = w.yn; P.yd[r] = w.yd; P.coef[r] = w.coef;
    }
    P.rows_e = c.nrows;
    P.lhs_e = c.lhs;
  }
  P.rows_pp = r;
  P.tile_terms = (uint32_t)(cfg.tile_terms > 0 ? cfg.tile_terms : (1 << 20));
  P.max_tiles = (uint32_t)(cfg.max_tiles > 0 ? cfg.max_tiles : 8);

  const size_t cap = cfg.chunk > 0 ? (size_t)cfg.chunk : kChunkPrimes;
  const uint32_t chunk = (uint32_t)(n < cap ? n : cap);
  const size_t nseg = (size_t)chunk * P.rows_pp;
  Scratch sc(s);
  uint32_t *u32tmp = nullptr, *scal = nullptr;
  WV_CHECK(sc.get(&P.ctx, chunk));
  WV_CHECK(sc.get(&P.flag, chunk));
  WV_CHECK(sc.get(&P.pos, chunk));
  WV_CHECK(sc.get(&P.seg_lo, nseg));
  WV_CHECK(sc.get(&P.seg_cnt, nseg));
  WV_CHECK(sc.get(&P.seg_tiles, nseg));
  WV_CHECK(sc.get(&P.seg_first, nseg));
  WV_CHECK(sc.get(&P.partials, nseg * P.max_tiles));
  WV_CHECK(sc.get(&u32tmp, scan_tmp_elems(nseg)));
  WV_CHECK(sc.get(&scal, 256));
  P.bk = scal + 64;
  P.n31 = scal + 0;
  P.total_tiles = scal + 1;
  P.split_tile = scal + 2;
  P.counters = scal + 4;

  for (size_t base = 0; base < n; base += chunk) {
    P.n = (uint32_t)((n - base) < chunk ? (n - base) : chunk);
    P.primes = d_primes + base;
    P.out_b = do_b ? d_out_b + base : nullptr;
    P.out_e = do_e ? d_out_e + base : nullptr;
    const unsigned gp = (P.n + 255) / 256;
    WV_CUDA(cudaMemsetAsync(P.bk, 0, 192 * sizeof(uint32_t), s));
    WV_LAUNCH("plan_prime", k_plan_prime, gp, 256, 0, s, P);
    WV_LAUNCH("plan_buckets", k_plan_buckets, 1, 32, 0, s, P);
    WV_LAUNCH("plan_scatter", k_plan_scatter, gp, 256, 0, s, P);
    const size_t ns = (size_t)P.n * P.rows_pp;
    WV_LAUNCH("plan_segments", k_plan_segments, (unsigned)((ns + 255) / 256), 256, 0, s, P);
    WV_CHECK(scan_exclusive_u32(P.seg_tiles, P.seg_first, ns, P.total_tiles, u32tmp, s));
    WV_LAUNCH("plan_split", k_plan_split, 1, 1, 0, s, P);
    WV_CHECK(launch_accumulate<false>(P, cfg, dev->sms, s));
    WV_CHECK(launch_accumulate<true>(P, cfg, dev->sms, s));
    const uint32_t nk = (do_b ? 1 : 0) + (do_e ? 1 : 0);
    const size_t warps = (size_t)P.n * nk;
    WV_LAUNCH("finalize", k_finalize, (unsigned)((warps * 32 + 255) / 256), 256, 0, s, P);
  }
  return WV_OK;
}

// ------------------------------------------------------------------ phases
// The launch sequence of residues_device split into its phases, for callers
// that interleave the accumulation of several prime lists (the serving loop):
// plan_build -> plan_totals -> epoch_launch (any number of times, over any
// tile ranges) -> plan_finalize -> plan_free.

static void fill_rows(Plan &P, const ResidueConfig &cfg) {
  uint32_t r = 0;
  if (cfg.cong_b >= 0) {
    const WvCongruence &c = kWvCongruences[cfg.cong_b];
    for (int j = 0; j < c.nrows; ++j, ++r) {
      const WvRow &w = kWvRows[c.row_offset + j];
      P.xn[r] = w.xn; P.xd[r] = w.xd; P.yn[r] = w.yn; P.yd[r] = w.yd; P.coef[r] = w.coef;
    }
    P.rows_b = c.nrows;
    P.lhs_b = c.lhs;
  }
  if (cfg.cong_e >= 0) {
    const WvCongruence &c = kWvCongruences[cfg.cong_e];
    for (int j = 0; j < c.nrows; ++j, ++r) {
      const WvRow &w = kWvRows[c.row_offset + j];
      P.xn[r] = w.xn; P.xd[r] = w.xd; P.yn[r] = w.yn; P.yd[r] = w.yd; P.coef[r] = w.coef;
    }
    P.rows_e = c.nrows;
    P.lhs_e = c.lhs;
  }
  P.rows_pp = r;
  P.tile_terms = (uint32_t)(cfg.tile_terms > 0 ? cfg.tile_terms : (1 << 20));
  P.max_tiles = (uint32_t)(cfg.max_tiles > 0 ? cfg.max_tiles : 8);
}

static size_t rows_of(const ResidueConfig &cfg) {
  size_t r = 0;
  if (cfg.cong_b >= 0) r += kWvCongruences[cfg.cong_b].nrows;
  if (cfg.cong_e >= 0) r += kWvCongruences[cfg.cong_e].nrows;
  return r;
}

size_t plan_bytes(uint32_t n, const ResidueConfig &cfg) {
  const size_t ns = (size_t)n * rows_of(cfg);
  const size_t mt = cfg.max_tiles > 0 ? cfg.max_tiles : 8;
  return n * (sizeof(PrimeCtx) + 8) + ns * (8 + 8 + 4 + 4) + ns * mt * sizeof(ulonglong2) +
         scan_tmp_elems(ns) * 4 + 1024 + 16 * 256;
}

size_t plan_struct_bytes() { return sizeof(Plan); }

wv_status plan_build(const uint64_t *d_primes, uint32_t n, const ResidueConfig &cfg, PlanState *ps,
                     cudaStream_t s) {
  if (n == 0 || n > 65536) return set_error(WV_EINVAL, "plan_build: n=%u not in [1, 65536]", n);
  ps->host = new Plan();
  Plan &P = *ps->host;
  memset(&P, 0, sizeof P);
  fill_rows(P, cfg);
  const size_t ns = (size_t)n * P.rows_pp;
  auto get = [&](void **p, size_t bytes) -> wv_status {
    WV_CHECK(scratch_alloc(p, bytes + 256, s));
    ps->blocks[ps->nblocks++] = *p;
    ps->bytes += bytes + 256;
    return WV_OK;
  };
  uint32_t *u32tmp = nullptr, *scal = nullptr;
  WV_CHECK(get((void **)&P.ctx, n * sizeof(PrimeCtx)));
  WV_CHECK(get((void **)&P.flag, n * 4));
  WV_CHECK(get((void **)&P.seg_lo, ns * 8));
  WV_CHECK(get((void **)&P.seg_cnt, ns * 8));
  WV_CHECK(get((void **)&P.seg_tiles, ns * 4));
  WV_CHECK(get((void **)&P.seg_first, ns * 4));
  WV_CHECK(get((void **)&P.partials, ns * P.max_tiles * sizeof(ulonglong2)));
  WV_CHECK(get((void **)&u32tmp, scan_tmp_elems(ns) * 4));
  WV_CHECK(get((void **)&scal, 1024));
  P.pos = nullptr;
  P.bk = scal + 64;
  P.n31 = scal + 0;
  P.total_tiles = scal + 1;
  P.split_tile = scal + 2;
  P.counters = scal + 4;
  P.n = n;
  P.primes = d_primes;
  ps->n = n;
  const unsigned gp = (n + 255) / 256;
  WV_CUDA(cudaMemsetAsync(P.bk, 0, 192 * sizeof(uint32_t), s));
  WV_LAUNCH("plan_prime", k_plan_prime, gp, 256, 0, s, P);
  WV_LAUNCH("plan_buckets", k_plan_buckets, 1, 32, 0, s, P);
  WV_LAUNCH("plan_scatter", k_plan_scatter, gp, 256, 0, s, P);
  WV_LAUNCH("plan_segments", k_plan_segments, (unsigned)((ns + 255) / 256), 256, 0, s, P);
  WV_CHECK(scan_exclusive_u32(P.seg_tiles, P.seg_first, ns, P.total_tiles, u32tmp, s));
  WV_LAUNCH("plan_split", k_plan_split, 1, 1, 0, s, P);
  return WV_OK;
}

wv_status plan_totals(PlanState *ps, cudaStream_t s) {
  uint32_t v[3] = {0, 0, 0};
  WV_CUDA(cudaMemcpyAsync(v, ps->host->n31, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  WV_CUDA(cudaStreamSynchronize(s));
  ps->total = v[1];
  ps->split = v[2];
  return WV_OK;
}

wv_status plan_upload(const PlanState *ps, Plan *d_plan, cudaStream_t s) {
  WV_CUDA(cudaMemcpyAsync(d_plan, ps->host, sizeof(Plan), cudaMemcpyHostToDevice, s));
  return WV_OK;
}

wv_status epoch_launch(bool wide, const EpochItem *d_items, uint32_t n_items, uint32_t total,
                       const Plan *d_plans, uint32_t *d_counter, const ResidueConfig &cfg, int sms,
                       cudaStream_t s) {
  if (total == 0) return WV_OK;
  void (*kern)(const EpochItem *, uint32_t, uint32_t, const Plan *, uint32_t *) =
      wide ? (cfg.ilp == 1 ? k_epoch<true, 1, 9> : k_epoch<true, 2, 9>)
           : (cfg.ilp == 1 ? k_epoch<false, 1, 9> : k_epoch<false, 2, 9>);
  int occ = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAccThreads, 0));
  if (occ < 1) occ = 1;
  WV_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s));
  WV_LAUNCH(wide ? "epoch_m64" : "epoch_m31", kern, (unsigned)(sms * occ), kAccThreads, 0, s,
            d_items, n_items, total, d_plans, d_counter);
  return WV_OK;
}

wv_status epoch_launch_mixed(const EpochItem *d_items, uint32_t n_items, uint32_t total,
                             const Plan *d_plans, uint32_t *d_counter, const ResidueConfig &cfg,
                             int sms, int reserve_blocks, cudaStream_t s) {
  if (total == 0) return WV_OK;
  void (*kern)(const EpochItem *, uint32_t, uint32_t, const Plan *, uint32_t *) =
      cfg.ilp == 1 ? k_epoch_mixed<1> : k_epoch_mixed<2>;
  int occ = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAccThreads, 0));
  if (occ < 1) occ = 1;
  WV_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s));
  int grid = sms * occ - reserve_blocks;
  if (grid < 1) grid = 1;
  WV_LAUNCH("epoch", kern, (unsigned)grid, kAccThreads, 0, s, d_items, n_items, total, d_plans,
            d_counter);
  return WV_OK;
}

wv_status plan_finalize(PlanState *ps, uint64_t *d_out_b, uint64_t *d_out_e, cudaStream_t s) {
  Plan P = *ps->host;
  P.out_b = P.rows_b ? d_out_b : nullptr;
  P.out_e = P.rows_e ? d_out_e : nullptr;
  const uint32_t nk = (P.rows_b ? 1u : 0u) + (P.rows_e ? 1u : 0u);
  const size_t warps = (size_t)P.n * nk;
  WV_LAUNCH("finalize", k_finalize, (unsigned)((warps * 32 + 255) / 256), 256, 0, s, P);
  return WV_OK;
}

void plan_free(PlanState *ps, cudaStream_t s) {
  for (int i = ps->nblocks - 1; i >= 0; --i) scratch_free(ps->blocks[i], s);
  ps->nblocks = 0;
  ps->bytes = 0;
  delete ps->host;
  ps->host = nullptr;
}

// ------------------------------------------------------------------ no-alloc
// Residues without any allocation: every scratch buffer of the launch sequence
// above is carved from one file-scope device array of fixed size instead of
// the library's stream-ordered pool.  Sized for kNoAllocMaxPrimes primes per
// call with the default congruences and launch shape (max_tiles 8).
constexpr uint32_t kNoAllocMaxPrimes = 1024;
constexpr uint32_t kNoAllocTiles = 8;

__host__ __device__ constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaSegs = (size_t)kNoAllocMaxPrimes * kMaxRowsPP;
constexpr size_t kNaScanTmp = kNaSegs / 4096 + 2;  // scan_tmp_elems bound for kNaSegs
constexpr size_t kNaBytes =
    na_align(kNoAllocMaxPrimes * sizeof(PrimeCtx)) + 2 * na_align(kNoAllocMaxPrimes * 4) +
    2 * na_align(kNaSegs * 8) + 2 * na_align(kNaSegs * 4) +
    na_align(kNaSegs * kNoAllocTiles * sizeof(ulonglong2)) + na_align(kNaScanTmp * 4) + 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

static std::mutex g_na_mu;
static void *g_na_addr[64];  // device address of g_noalloc_scratch, per device

wv_status residues_noalloc(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                           uint64_t *d_out_e, cudaStream_t s) {
  if (n == 0) return WV_OK;
  if (!d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  if (n > kNoAllocMaxPrimes)
    return set_error(WV_ERANGE, "wv_residues_pm3_noalloc takes at most %u primes per call (got %zu)",
                     kNoAllocMaxPrimes, n);
  const bool do_b = d_out_b != nullptr, do_e = d_out_e != nullptr;
  if (!do_b && !do_e) return WV_OK;
  int dev = 0;
  WV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(WV_EINVAL, "device index %d out of range", dev);
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
      // The array's name is only a host-side stand-in: its device address
      // must be looked up once per device, with that device current.
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
      g_na_addr[dev] = ptr;
    }
    base = (unsigned char *)g_na_addr[dev];
  }
  int sms = 0;
  WV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  ResidueConfig cfg;  // library defaults
  Plan P;
  memset(&P, 0, sizeof P);
  uint32_t r = 0;
  if (do_b) {
    const WvCongruence &c = kWvCongruences[cfg.cong_b];
    for (int j = 0; j < c.nrows; ++j, ++r) {
      const WvRow &w = kWvRows[c.row_offset + j];
      P.xn[r] = w.xn; P.xd[r] = w.xd; P.yn[r] = w.yn; P.yd[r] = w.yd; P.coef[r] = w.coef;
    }
    P.rows_b = c.nrows;
    P.lhs_b = c.lhs;
  }
  if (do_e) {
    const WvCongruence &c = kWvCongruences[cfg.cong_e];
    for (int j = 0; j < c.nrows; ++j, ++r) {
      const WvRow &w = kWvRows[c.row_offset + j];
      P.xn[r] = w.xn; P.xd[r] = w.xd; P.yn[r] = w.yn; P.yd[r] = w.yd; P.coef[r] = w.coef;
    }
    P.rows_e = c.nrows;
    P.lhs_e = c.lhs;
  }
  P.rows_pp = r;
  P.tile_terms = (uint32_t)cfg.tile_terms;
  P.max_tiles = kNoAllocTiles;
  // carve the scratch array
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char *q = base + off;
    off += na_align(bytes);
    return q;
  };
  P.ctx = (PrimeCtx *)carve(kNoAllocMaxPrimes * sizeof(PrimeCtx));
  P.flag = (uint32_t *)carve(kNoAllocMaxPrimes * 4);
  P.pos = (uint32_t *)carve(kNoAllocMaxPrimes * 4);
  P.seg_lo = (uint64_t *)carve(kNaSegs * 8);
  P.seg_cnt = (uint64_t *)carve(kNaSegs * 8);
  P.seg_tiles = (uint32_t *)carve(kNaSegs * 4);
  P.seg_first = (uint32_t *)carve(kNaSegs * 4);
  P.partials = (ulonglong2 *)carve(kNaSegs * kNoAllocTiles * sizeof(ulonglong2));
  uint32_t *u32tmp = (uint32_t *)carve(kNaScanTmp * 4);
  uint32_t *scal = (uint32_t *)carve(256 * sizeof(uint32_t));
  if (off > kNaBytes) return set_error(WV_EINVAL, "internal: no-alloc scratch layout overflow");
  P.bk = scal + 64;
  P.n31 = scal + 0;
  P.total_tiles = scal + 1;
  P.split_tile = scal + 2;
  P.counters = scal + 4;  // zeroed by k_plan_split before every accumulation
  P.n = (uint32_t)n;
  P.primes = d_primes;
  P.out_b = do_b ? d_out_b : nullptr;
  P.out_e = do_e ? d_out_e : nullptr;

  const unsigned gp = (P.n + 255) / 256;
  const size_t ns = (size_t)P.n * P.rows_pp;
  WV_CUDA(cudaMemsetAsync(P.bk, 0, 192 * sizeof(uint32_t), s));
  k_plan_prime<<<gp, 256, 0, s>>>(P);
  k_plan_buckets<<<1, 32, 0, s>>>(P);
  k_plan_scatter<<<gp, 256, 0, s>>>(P);
  k_plan_segments<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(P);
  WV_CHECK(scan_exclusive_u32_bare(P.seg_tiles, P.seg_first, ns, P.total_tiles, u32tmp, s));
  k_plan_split<<<1, 1, 0, s>>>(P);
  WV_CUDA(cudaGetLastError());
  void (*k31)(Plan) = k_accumulate<false, 2, 9>;
  void (*k64)(Plan) = k_accumulate<true, 2, 1>;
  int occ31 = 0, occ64 = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ31, k31, kAccThreads, 0));
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k64, kAccThreads, 0));
  k31<<<(unsigned)(sms * (occ31 > 0 ? occ31 : 1)), kAccThreads, 0, s>>>(P);
  k64<<<(unsigned)(sms * (occ64 > 0 ? occ64 : 1)), kAccThreads, 0, s>>>(P);
  const size_t warps = (size_t)P.n * ((do_b ? 1 : 0) + (do_e ? 1 : 0));
  k_finalize<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(P);
  WV_CUDA(cudaGetLastError());
  return WV_OK;
}

}  // namespace wv

using namespace wv;

extern "C" {

wv_status wv_residues_ex(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                         uint64_t *d_out_e, const wv_options *opt, wv_stream stream) {
  clear_error();
  if (n > 0 && !d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  if (n > ((size_t)1 << 40)) return set_error(WV_EINVAL, "n too large");
  ResidueConfig cfg;
  WV_CHECK(resolve_config(opt, d_out_b != nullptr, d_out_e != nullptr, &cfg));
  return residues_device(d_primes, n, d_out_b, d_out_e, cfg, (cudaStream_t)stream);
}

wv_status wv_residues_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                          uint64_t *d_out_e, wv_stream stream) {
  return wv_residues_ex(d_primes, n, d_out_b, d_out_e, nullptr, stream);
}

wv_status wv_bernoulli_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out, wv_stream stream) {
  if (n > 0 && !d_out) {
    clear_error();
    return set_error(WV_EINVAL, "d_out is NULL");
  }
  return wv_residues_ex(d_primes, n, d_out, nullptr, nullptr, stream);
}

wv_status wv_residues_pm3_noalloc(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                                  uint64_t *d_out_e, wv_stream stream) {
  clear_error();
  return residues_noalloc(d_primes, n, d_out_b, d_out_e, (cudaStream_t)stream);
}

wv_status wv_euler_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out, wv_stream stream) {
  if (n > 0 && !d_out) {
    clear_error();
    return set_error(WV_EINVAL, "d_out is NULL");
  }
  return wv_residues_ex(d_primes, n, nullptr, d_out, nullptr, stream);
}

}  // extern "C"
