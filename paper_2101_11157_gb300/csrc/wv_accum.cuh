// wv_accum.cuh -- steps a3-a5 on the device: term generation, accumulation
// of eqn 3.12 / eqn 3.14 per warp tile, and the lane/warp merge; the plan
// layout the planner fills; and the accumulation kernels as templates.
//
// The kernels are instantiated in four translation units that compile in
// parallel: wv_residue.cu (32-bit path), wv_acc_m64.cu (64-bit path),
// wv_acc_epoch.cu (the serving loop's epoch kernels) and wv_acc_m64x.cu
// (64-bit formulations kept for ablation).  The host side reaches them
// through the getters at the end.
#pragma once

#include "wv_arith.cuh"
#include "wv_internal.h"
#include "wv_tables.h"

namespace wv {

constexpr int kAccThreads = 256;
constexpr int kMaxRowsPP = 66;  // B rows + E rows of BB30 + EE33 (the allocation-free path)
constexpr int kMaxDist = 512;   // distinct coefficient bases d of one congruence
constexpr uint32_t kChunkPrimes = 16384;  // primes per internal launch sequence
constexpr uint64_t kGroupMinChain = 48;   // grouped path only for chains of >= 48 terms

struct Plan {
  uint32_t n;                   // primes in this chunk
  uint32_t check;               // nonzero: the planner verifies each input's primality
  uint32_t rows_b, rows_e, rows_pp;
  uint32_t tile_terms, max_tiles;
  const uint64_t *primes;       // caller's primes (chunk base)
  uint64_t *out_b, *out_e;      // caller's outputs (chunk base), may be null
  PrimeCtx *ctx;                // per slot (M31 slots first, then M64)
  uint32_t *flag, *pos, *n31;   // flag: p-bucket per prime; n31: slots with p < 2^31
  uint32_t *bk;                 // 3 x 64 words: bucket counts, offsets, cursors
  uint64_t *seg_lo, *seg_cnt;   // per segment (slot * rows_pp + row)
  uint32_t *seg_tiles, *seg_first;
  uint32_t *tile_seg;           // per tile: its segment (written by the planner)
  uint32_t *total_tiles, *split_tile;
  uint32_t *counters;           // [0] M31 accumulation, [1] M64 accumulation
  ulonglong2 *partials;         // per tile (c0, c1), canonical
  // congruence rows: rows [0, rows_b) are B rows, [rows_b, rows_pp) E rows,
  // taken from the registry (device copy): B row j is registry row rb0 + j,
  // E row j is re0 + j; a row's coefficient is sum_k c_k d_k^-ex with the
  // bases d of its congruence at cg_dist[db0 ..] (B) / [de0 ..] (E)
  const uint32_t *cg_rows;
  const int64_t *cg_tc;
  const uint16_t *cg_td;
  const uint64_t *cg_dist;
  uint32_t rb0, re0, db0, dbn, de0, den;
  uint32_t ex_b, ex_e;  // 3 / 2 for B_{p-3} / E_{p-3}; e at a general index
  int64_t lhs_b, lhs_e;
  // general index (0: the B_{p-3} / E_{p-3} forms): the exponent e of the
  // inverse-power sums, and (a, b, c) of C_k(a,b,c) for B
  uint32_t gen_e_b, gen_e_e;
  uint32_t glhs[3];
  // lane chains (lane != 0): a tile is one lane's piece of a segment, and a
  // warp runs 32 of them.  rec lists the pieces by class (32-bit signed /
  // unsigned / 64-bit path, B / E) and, inside a class, by rising length,
  // each class padded to whole warps; lane_w = {warps of the 32-bit kernel,
  // all warps}.  Pieces per segment come from the path's chain length
  // (terms at most per piece: from lane_sum = terms per path and the
  // targets below, or fixed by the host in lane_fix).
  uint32_t lane;
  struct PieceRec *rec;  // the sorted pieces (padding: tile = kNoChain)
  uint32_t *chain_key, *chain_hist, *lane_w;
  uint64_t *lane_sum;
  uint64_t lane_target[2], lane_min[2];  // chains wanted per path, shortest chain length
  uint64_t lane_fix[2];  // nonzero: the chain length per path, fixed by the host
  uint32_t uform_min[2];  // forms 48..50: pieces of at least this many terms take the u form
};
constexpr uint32_t kNoChain = 0xffffffffu;
// One lane chain as the planner lists it, in sorted order, so that a warp's
// 32 lanes read their pieces with one coalesced load: the first term s, the
// number of terms, the tile (the slot of its partial), the prime's slot and
// the row (B rows first).
struct PieceRec {
  uint64_t start;
  uint32_t n, tile, slot, row;
};

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

// Unsigned 32-bit words: wide products and word access in PTX.
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

// 2^30 <= p < 2^31: unsigned 32-bit Montgomery with R' = 2^32 and canonical
// values in [0, p).  A product a b < p^2 < 2^62 plus m p < 2^63 stays below
// 2^64, and (a b + m p) / 2^32 < 1.5 p, so one conditional subtraction makes
// it canonical; sums of two products (< 2 p^2) reduce below 2 p the same way.
// The constants of R' (R' mod p, R'^2 mod p) are formed here, once per chain,
// since the context of such a prime carries those of R = 2^64.
struct U31Set {
  uint32_t up, qn;               // p, -p^-1 mod 2^32
  uint32_t one, r2, c1, c2, c6;  // R', R'^2 mod p; the plain constants 1, 2, 6
  __device__ __forceinline__ explicit U31Set(const PrimeCtx &c)
      : up((uint32_t)c.p), qn(0u - (uint32_t)c.q), c1(1u), c2(2u), c6(6u) {
    one = (uint32_t)((1ull << 32) % c.p);
    r2 = (uint32_t)(((uint64_t)one * one) % c.p);
  }
  __device__ __forceinline__ uint32_t redc(uint64_t w) const {  // w < 2^63: w R'^-1, < 2 p in, [0, p) out
    const uint32_t m = ulo(w) * qn;
    const uint32_t t = uhi(umad_wide(m, up, w));
    return min(t, t - up);
  }
  __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const {  // a b R'^-1
    return redc(umul_wide(a, b));
  }
  __device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b) const {  // a b
    return mul(mul(a, b), r2);
  }
  __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) const {
    const uint32_t x = a + b;
    return min(x, x - up);
  }
  __device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b) const {
    const uint32_t x = a - b;
    return min(x, x + up);
  }
};

// p < 2^30: signed 32-bit Montgomery, R = 2^32.  AR selects the product
// formulation: 1 = hi(c t) and lo(c tq) with tq = t p^-1 shared by c0 and c1;
// 2 = the full 64-bit product c t (one wide multiply) and m = lo(c t) p^-1.
template <int ILP, bool CUBES, int AR, bool LANE = false>
__device__ __forceinline__ void tile_m31(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                         int64_t &r0, int64_t &r1) {
  const int lane = threadIdx.x & 31;
  const int32_t p = (int32_t)ctx.p;
  const uint32_t up = (uint32_t)ctx.p;
  const uint32_t q = (uint32_t)ctx.q;
  const uint64_t nch = LANE ? ILP : 32 * ILP;  // lane chains: the lane owns the tile
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  int32_t c0[ILP], c1[ILP], t[ILP], d1[ILP], d2[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = LANE ? k : k * 32 + lane;
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
    if ((uint32_t)(LANE ? k : k * 32 + lane) < rem) step(k, z);

  const Mont M(ctx);
  int64_t a0 = m31_canon(c0[0], p), a1 = m31_canon(c1[0], p);
#pragma unroll
  for (int k = 1; k < ILP; ++k) M.combine(a0, a1, m31_canon(c0[k], p), m31_canon(c1[k], p));
  if (!LANE) warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

template <bool U> struct SetOf { using T = M31Set; };
template <> struct SetOf<true> { using T = U31Set; };

// ---- grouped accumulation (p < 2^31) ------------------------------------
// eqn 3.14 applied to a GROUP of K consecutive terms: the group's factor
// prod_{i<K} (z + (s+i)^e) = G0(s) + G1(s) z + O(z^2) with
//   G0(s) = prod_i (s+i)^e,   G1(s) = sum_i prod_{j!=i} (s+j)^e,
// polynomials in s of degree K e and (K-1) e.  Both are stepped s -> s+K by
// forward differences (additions only), and each group costs three products:
//   c0 <- c0 G0,   c1 <- c1 G0 + c0 G1.
// The tables are built so that G0 and R G1 carry the same power of R; as in
// the single-term step the ratio c1/c0 then accumulates R * sum t^-1.
//
// NF of the table additions per group (the G0 table's from the low order up,
// then G1's) are written as an inline PTX block whose a + b - p is a
// three-input add, which only the integer ALU executes.  The others are
// plain C; the compiler may place their two-input adds on the multiply pipe,
// which the products already fill.  NF moves work from that pipe to the ALU.

template <int ILP, bool CUBES, int AR, int NF = 0, int KG = 0, bool U = false, bool LANE = false,
          bool UF = false>
__device__ __forceinline__ void tile_m31_grouped(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                                 int64_t &r0, int64_t &r1) {
  // U: the unsigned form for 2^30 <= p < 2^31 (U31Set), run by the same
  // kernel; its chains end with c1 scaled from R' = 2^32 to the context's
  // R = 2^64 before the lanes merge
  using SetT = typename SetOf<U>::T;
  const SetT S(ctx);
  constexpr int K = KG ? KG : (CUBES ? 2 : 3);  // terms per group (default 2 cubes / 3 squares)
  constexpr int EX = CUBES ? 3 : 2;    // t = s^EX
  constexpr int DA = K * EX;           // degree of G0
  constexpr int DB = (K - 1) * EX;     // degree of G1
  // UF: G0 = u^EX with u = prod_{i<K} (s+i), so the first table is u's, of
  // degree K, and each group forms G0 with EX - 1 products from it
  constexpr int DT = UF ? K : DA;            // degree of the first table
  constexpr int DTOP = DT > DB ? DT : DB;    // points of the set-up: 0 .. DTOP
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  const int32_t p = (int32_t)ctx.p;
  const uint32_t up = (uint32_t)ctx.p;
  const uint32_t q = (uint32_t)ctx.q;
  const uint32_t uz = (AR >= 7) ? 0u : (ctx.flags >> 16);  // runtime zero (AR 5: three-input adds)
  const int32_t np = -p;
  const uint64_t nch = LANE ? ILP : 32 * ILP;  // lane chains: the lane owns the tile
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  const uint64_t G = len / K;  // groups per chain, the same for every lane
  int32_t c0[ILP], c1[ILP], ga[ILP][DT + 1], gb[ILP][DB + 1];
  uint64_t s_tail[ILP];
  uint32_t n_tail[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = LANE ? k : k * 32 + lane;
    const uint64_t s = start + ch * len + (ch < rem ? ch : rem);
    const uint64_t L = len + (ch < rem ? 1 : 0);
    s_tail[k] = s + G * K;
    n_tail[k] = (uint32_t)(L - G * K);
    // Difference tables of G0 and G1 at s, s + K, ..., s + DA K, as on the
    // 64-bit path: each point's pair from the plain powers t = x^e of its K
    // consecutive x by P <- REDC(P t), Q <- REDC(Q t) + P (start P = t,
    // Q = R), which gives G0 = R^-(K-1) prod t_i and G1 = R^-(K-2) sum_i
    // prod_{j != i} t_j -- the common factor R^-(K-1) on G0 and R G1 leaves
    // c1 / c0 unchanged; points from the top down (x^e by backward
    // differences), folded into the diagonals: e_j <- (-1)^j D^j.
    {
      // 32-bit residues in [0, p) throughout (p < 2^31); s < p, so the top
      // point needs at most one subtraction of p
      // 32-bit residues in [0, p) (S: the chain's Montgomery set, above)
      uint64_t x64 = s + (uint64_t)(K * (DTOP + 1) - 1);
      x64 = x64 >= ctx.p ? (x64 >= 2 * ctx.p ? x64 % ctx.p : x64 - ctx.p) : x64;
      const uint32_t xr = (uint32_t)x64;
      const uint32_t sq = S.mulmod(xr, xr);
      const uint32_t x2 = S.add(xr, xr);
      uint32_t t, d1, d2;
      if (EX == 3) {  // x^3, 3x^2 - 3x + 1, 6x - 6, 6
        t = S.mulmod(sq, xr);
        d1 = S.sub(S.add(S.add(S.add(sq, sq), sq), S.c1), S.add(x2, xr));
        d2 = S.sub(S.add(S.add(x2, xr), S.add(x2, xr)), S.c6);
      } else {        // x^2, 2x - 1, 2
        t = sq;
        d1 = S.sub(x2, S.c1);
        d2 = S.c2;
      }
      uint32_t va[DT + 1], vb[DB + 1];
      uint32_t xc = xr;  // the plain x of the current term (UF: u's factors)
#pragma unroll
      for (int i = 0; i <= DT; ++i) va[i] = 0;
#pragma unroll
      for (int i = 0; i <= DB; ++i) vb[i] = 0;
      // the point loop stays rolled (it runs once per chain; unrolled it is
      // kilobytes of code that short tiles fetch again and again); the table
      // indices stay compile-time, the diagonal lengths are predicated
      // (signed words, p < 2^30) the point's products as the main loop's
      // REDC folded into a wide multiply-add, not canonicalised: from t in
      // [0, p), P and Pu stay in (-p, p) and Q in (-2p, 2p); u's factor x
      // steps as a plain integer (it falls by at most K (DTOP + 1) < 2^10
      // below 0); one canonicalisation per point before the fold
      const int32_t sp = (int32_t)ctx.p;
      auto sredc = [&](int32_t a, int32_t b) {
        const int64_t w = mul_wide(a, b);
        return hi32(mad_wide((int32_t)((uint32_t)lo32(w) * q), np, w));
      };
      int32_t xs = (int32_t)xc;
#pragma unroll 1
      for (int m = DTOP; m >= 0; --m) {
        uint32_t P = 0, Q = S.one, Pu = 0;
        if constexpr (!U) {
          int32_t Ps = 0, Qs = (int32_t)S.one, Pus = 0;
#pragma unroll
          for (int i = 0; i < K; ++i) {
            if (i == 0) {
              Ps = (int32_t)t;
              if (UF) Pus = xs;
            } else {
              Qs = sredc(Qs, (int32_t)t) + Ps;
              Ps = sredc(Ps, (int32_t)t);
              if (UF) Pus = sredc(Pus, xs);
            }
            t = S.sub(t, d1);
            d1 = S.sub(d1, d2);
            if (EX == 3) d2 = S.sub(d2, S.c6);
            if (UF) xs -= 1;
          }
          P = (uint32_t)m31_canon(Ps, sp);
          Q = (uint32_t)m31_canon(Qs, sp);
          if (UF) Pu = (uint32_t)m31_canon(Pus, sp);
        } else {
#pragma unroll
          for (int i = 0; i < K; ++i) {
            if (i == 0) {
              P = t;
              if (UF) Pu = xc;
            } else {
              Q = S.add(S.mul(Q, t), P);
              P = S.mul(P, t);
              if (UF) Pu = S.mul(Pu, xc);
            }
            t = S.sub(t, d1);
            d1 = S.sub(d1, d2);
            if (EX == 3) d2 = S.sub(d2, S.c6);
            if (UF) xc = S.sub(xc, S.c1);
          }
        }
        // fold the point into the diagonals over their whole length: with
        // zeros before the first point, a difference of order j <= D at the
        // last point still involves only its last j + 1 (real) points
        if (m <= DT) {
          uint32_t nv = UF ? Pu : P;
#pragma unroll
          for (int j = 0; j <= DT; ++j) {
            const uint32_t old = va[j];
            va[j] = nv;
            if (j < DT) nv = S.sub(nv, old);
          }
        }
        if (m <= DB) {
          uint32_t nv = Q;
#pragma unroll
          for (int j = 0; j <= DB; ++j) {
            const uint32_t old = vb[j];
            vb[j] = nv;
            if (j < DB) nv = S.sub(nv, old);
          }
        }
      }
#pragma unroll
      for (int j = 0; j <= DT; ++j) ga[k][j] = (int32_t)((j & 1) ? S.sub(0, va[j]) : va[j]);
#pragma unroll
      for (int j = 0; j <= DB; ++j) gb[k][j] = (int32_t)((j & 1) ? S.sub(0, vb[j]) : vb[j]);
    }
    c0[k] = (int32_t)S.one;
    c1[k] = 0;
  }
  auto modadd = [&](int32_t &a, int32_t b) {
    const uint32_t x = (uint32_t)a + (uint32_t)b + uz;
    const uint32_t y = (uint32_t)a + (uint32_t)b - up;
    a = (int32_t)min(x, y);
  };
  // the same modular add as one PTX block: a - p + b (a three-input add once
  // fused), a + b and their unsigned minimum; opaque to the front end, so
  // the two sums are not merged into a shared a + b
  auto modadd_alu = [&](int32_t &a, int32_t b) {
    uint32_t r;
    asm("{\n\t.reg .u32 t;\n\t"
        "add.u32 t, %1, %3;\n\t"
        "add.u32 t, t, %2;\n\t"
        "add.u32 %0, %1, %2;\n\t"
        "min.u32 %0, %0, t;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)a), "r"((uint32_t)b), "r"((uint32_t)np));
    a = (int32_t)r;
  };
  const uint32_t G32 = (uint32_t)G;  // chains hold fewer than 2^32 groups (tiles < 2^32 terms)
  // two groups per loop trip: the trip's counter, compare and branch are
  // about 3 % of a group's instructions (unrolling the 64-bit kernel's loop
  // the same way measured 0.6 % slower)
#pragma unroll 2
  for (uint32_t g = 0; g < G32; ++g) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
      int32_t A;
      if constexpr (UF && U) {
        // G0 = u^EX from the u table's value, canonical
        const uint32_t Uv = (uint32_t)ga[k][0], U2 = S.mul(Uv, Uv);
        A = (int32_t)(EX == 3 ? S.mul(U2, Uv) : U2);
      } else if constexpr (UF) {
        // the same on signed words, REDC folded into a wide multiply-add: from
        // u in [0, p) the square lies in (-3p/4, 3p/4) and the cube in (-p, p),
        // inside the accumulator's operand range
        const int32_t Uv = ga[k][0];
        const int64_t w2 = mul_wide(Uv, Uv);
        const int32_t U2 = hi32(mad_wide((int32_t)((uint32_t)lo32(w2) * q), np, w2));
        if (EX == 3) {
          const int64_t w3 = mul_wide(U2, Uv);
          A = hi32(mad_wide((int32_t)((uint32_t)lo32(w3) * q), np, w3));
        } else {
          A = U2;
        }
      } else {
        A = ga[k][0];
      }
      const int32_t B = gb[k][0];
      if constexpr (U) {
        // the same with unsigned words: c0 G0 and c1 G0 + c0 G1 stay below
        // 2 p^2 < 2^63, and one subtraction makes each result canonical
        const uint64_t w0 = umul_wide((uint32_t)c0[k], (uint32_t)A);
        const uint64_t w1 = umad_wide((uint32_t)c0[k], (uint32_t)B, umul_wide((uint32_t)c1[k], (uint32_t)A));
        c0[k] = (int32_t)S.redc(w0);
        c1[k] = (int32_t)S.redc(w1);
      } else if (AR >= 7) {
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
      for (int j = 0; j < DT; ++j) {
        if (j < NF) modadd_alu(ga[k][j], ga[k][j + 1]);
        else modadd(ga[k][j], ga[k][j + 1]);
      }
#pragma unroll
      for (int j = 0; j < DB; ++j) {
        if (DT + j < NF) modadd_alu(gb[k][j], gb[k][j + 1]);
        else modadd(gb[k][j], gb[k][j + 1]);
      }
    }
  }
  if constexpr (UF) {
    // u^EX carries R^-(EX-1)K more than the G0 of the pair tables, so the
    // groups' ratio c1 / c0 is R^((EX-1)K) too large: scale c1 back once,
    // by a product with R^(1-(EX-1)K), before the single-term tail
    uint32_t f = S.one;
#pragma unroll 1
    for (int i = 0; i < (EX - 1) * K; ++i) f = S.mul(f, S.c1);
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
      const uint32_t c = U ? (uint32_t)c1[k] : (uint32_t)m31_canon(c1[k], p);
      c1[k] = (int32_t)S.mul(c, f);
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
        if constexpr (U) {  // c1 <- c1 t R'^-1 + c0, c0 <- c0 t R'^-1 (eqn 3.12), canonical
          const uint32_t n1 = S.add(S.mul((uint32_t)c1[k], (uint32_t)t), (uint32_t)c0[k]);
          c0[k] = (int32_t)S.mul((uint32_t)c0[k], (uint32_t)t);
          c1[k] = (int32_t)n1;
          continue;
        }
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
  // canonical pairs whose ratio c1 / c0 is R S (R of the context: for U the
  // chains carry R' S = 2^32 S, so c1 is multiplied by 2^32 mod p)
  auto canon = [&](int32_t v) -> int64_t {
    return U ? (int64_t)(uint32_t)v : m31_canon(v, p);
  };
  auto canon1 = [&](int32_t v) -> int64_t {
    return U ? (int64_t)((((uint64_t)(uint32_t)v) << 32) % ctx.p) : m31_canon(v, p);
  };
  int64_t a0 = canon(c0[0]), a1 = canon1(c1[0]);
#pragma unroll
  for (int k = 1; k < ILP; ++k) M.combine(a0, a1, canon(c0[k]), canon1(c1[k]));
  if (!LANE) warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// 2^30 <= p < 2^37: signed 64-bit Montgomery, R = 2^64.
template <int ILP, bool CUBES, bool LANE = false>
__device__ __forceinline__ void tile_m64(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                         int64_t &r0, int64_t &r1) {
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  const int64_t p = (int64_t)ctx.p;
  const uint64_t up = ctx.p;
  const uint64_t q = ctx.q;
  const uint64_t nch = LANE ? ILP : 32 * ILP;  // lane chains: the lane owns the tile
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  int64_t c0[ILP], c1[ILP], t[ILP], d1[ILP], d2[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = LANE ? k : k * 32 + lane;
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
    if ((uint32_t)(LANE ? k : k * 32 + lane) < rem) step(k);

  int64_t a0 = m64_canon(c0[0], p), a1 = m64_canon(c1[0], p);
#pragma unroll
  for (int k = 1; k < ILP; ++k) M.combine(a0, a1, m64_canon(c0[k], p), m64_canon(c1[k], p));
  if (!LANE) warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// ---- grouped accumulation for 2^30 <= p < 2^37 ------------------------------
// Montgomery with R = 2^64 done as two 32-bit rounds on unsigned words:
// p = p0 + p1 2^32 (p1 < 32), q = -p^-1 mod 2^32.  A product T = c g is held
// as a low word T0 and a 64-bit rest TY (T = T0 + TY 2^32); each round adds
// m p with m = (low word) q, which clears the low word exactly.  For
// c < p + 2^31 and g < 2^57 every intermediate fits its word and the result
// is below p + 2^31 (one conditional subtraction makes it canonical).
//
// The grouped scheme of the 32-bit path is used with larger groups here (8
// cubes, 12 squares): the
// group polynomials G0, G1 are stepped with plain 64-bit additions and no
// reduction, and every BLK groups the tables are brought back below 6 p by an
// approximate Barrett step (quotient from the high word times floor(2^62 / p),
// m64_shrink_q; the earlier, longer form m64_shrink leaves them below 10 p).
// Starting below 10 p, entry j of a degree-D table grows over B steps to at
// most 10 p sum_{i <= D-j} C(B, i) <= 10 p 2^B, so with BLK = 16 every entry
// stays below 10 p 2^16 < 2^57 (p < 2^37), whatever D.
//
// The scheme is parametrised by the group sizes (KB terms per group for the
// cubes of the Bernoulli sums, KE for the squares of the Euler sums), the
// shrink interval BLK and flags: 4 and 8 write (part of) the table additions
// as PTX carry chains (M64Split below), 16 selects the four-step shrink, 32
// the rolled per-chain set-up.
// A group costs the same 41 multiply-pipe slots whatever K, so larger groups
// cut the products per term; the tables cost 2 (D_A + D_B) additions per
// group and registers, which bound K.

struct M64K {
  uint32_t p0, p1, q, mhi;  // mhi = floor(2^62 / p)
  uint64_t p;
};

// (T0 + TY 2^32) 2^-64 mod p for T < 2^96, result below p + 2^32
__device__ __forceinline__ uint64_t m64_redc2(uint32_t T0, uint64_t TY, const M64K &K) {
  const uint32_t m0 = T0 * K.q;
  const uint64_t A = umad_wide(m0, K.p0, (uint64_t)T0);       // low word is 0
  const uint64_t U = umad_wide(m0, K.p1, TY) + uhi(A);        // (T + m0 p) / 2^32
  const uint32_t m1 = ulo(U) * K.q;
  const uint64_t B = umad_wide(m1, K.p0, (uint64_t)ulo(U));   // low word is 0
  return umad_wide(m1, K.p1, (uint64_t)uhi(U)) + uhi(B);      // (U + m1 p) / 2^32
}
// (T0 + TY 2^32) 2^-32 mod p for T < 2^96: one round, result below T / 2^32 + p
__device__ __forceinline__ uint64_t m64_redc1(uint32_t T0, uint64_t TY, const M64K &K) {
  const uint32_t m0 = T0 * K.q;
  const uint64_t A = umad_wide(m0, K.p0, (uint64_t)T0);  // low word is 0
  return umad_wide(m0, K.p1, TY) + uhi(A);               // (T + m0 p) / 2^32
}
// T = c g as (T0, TY); c < p + 2^31, g < 2^57
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

// v < 2^58  ->  v' = v (mod p) with v' < 6 p, in four multiply-pipe steps: the
// quotient q = hi(4 hi(v) floor(2^62 / p)) is at most floor(v / p) and short
// of it by less than 5.25, and v - q p is formed modulo 2^64 (where it is
// exact) as v + q (2^64 - p): one wide multiply-add for the low word of
// 2^64 - p, one low multiply-add into the high word for its high word.
__device__ __forceinline__ uint64_t m64_shrink_q(uint64_t v, const M64K &K, uint32_t np0,
                                                 uint32_t np1) {
  const uint32_t q = __umulhi(uhi(v) << 2, K.mhi);
  const uint64_t r = umad_wide(q, np0, v);
  return upack(ulo(r), uhi(r) + q * np1);
}

// group sizes, shrink interval and flags of each 64-bit formulation (arith)
template <int AR> struct M64Form {  // 9: the default
  static constexpr int KB = 8, KE = 12, BLK = 16, V = 16 | 32;
};
// 32..36: form 9 with its 64-bit table additions written as PTX carry chains
// (add.cc / addc on the two words) for a share of the entries, in quarters
// of the table (NFQ = 4: all), taken from the low order up.  Flag 4: the plain
// carry chain; flag 8: a runtime zero added into the high word as well, which
// makes that word's add a three-input add with carry in -- an instruction
// only the integer ALU has, so the entry stays off the multiply pipe.
template <int AR> struct M64Split { static constexpr int NFQ = 0; };
template <> struct M64Form<32> : M64Form<9> { static constexpr int V = 4 | 16 | 32; };
template <> struct M64Form<33> : M64Form<9> { static constexpr int V = 8 | 16 | 32; };
template <> struct M64Form<34> : M64Form<9> { static constexpr int V = 8 | 16 | 32; };
template <> struct M64Form<35> : M64Form<9> { static constexpr int V = 8 | 16 | 32; };
template <> struct M64Form<36> : M64Form<9> { static constexpr int V = 8 | 16 | 32; };
template <> struct M64Split<32> { static constexpr int NFQ = 4; };
template <> struct M64Split<33> { static constexpr int NFQ = 4; };
template <> struct M64Split<34> { static constexpr int NFQ = 2; };
template <> struct M64Split<35> { static constexpr int NFQ = 1; };
template <> struct M64Split<36> { static constexpr int NFQ = 3; };
// 37: form 9 with the earlier shrink (m64_shrink: a wide quotient, a 64-bit
// product and a 64-bit subtraction) in place of the four-step one (flag 16)
template <> struct M64Form<37> : M64Form<9> { static constexpr int V = 32; };
// 38: form 9 with its per-chain set-up loop unrolled, as it was (flag 32 off)
template <> struct M64Form<38> : M64Form<9> { static constexpr int V = 16; };

// a += b (64-bit) as an explicit carry chain over the two 32-bit words
__device__ __forceinline__ void add64_cc(uint64_t &a, uint64_t b) {
  asm("{\n\t.reg .u32 a0, a1, b0, b1;\n\t"
      "mov.b64 {a0, a1}, %0;\n\t"
      "mov.b64 {b0, b1}, %1;\n\t"
      "add.cc.u32 a0, a0, b0;\n\t"
      "addc.u32 a1, a1, b1;\n\t"
      "mov.b64 %0, {a0, a1};\n\t}"
      : "+l"(a)
      : "l"(b));
}
// the same with the runtime zero z added into the high word
__device__ __forceinline__ void add64_cc_z(uint64_t &a, uint64_t b, uint32_t z) {
  asm("{\n\t.reg .u32 a0, a1, b0, b1;\n\t"
      "mov.b64 {a0, a1}, %0;\n\t"
      "mov.b64 {b0, b1}, %1;\n\t"
      "add.cc.u32 a0, a0, b0;\n\t"
      "addc.u32 a1, a1, b1;\n\t"
      "add.u32 a1, a1, %2;\n\t"
      "mov.b64 %0, {a0, a1};\n\t}"
      : "+l"(a)
      : "l"(b), "r"(z));
}
template <> struct M64Form<12> { static constexpr int KB = 2, KE = 3, BLK = 8, V = 16 | 32; };
template <> struct M64Form<13> { static constexpr int KB = 3, KE = 4, BLK = 16, V = 16 | 32; };
template <> struct M64Form<14> { static constexpr int KB = 4, KE = 5, BLK = 16, V = 16 | 32; };
template <> struct M64Form<15> { static constexpr int KB = 5, KE = 6, BLK = 16, V = 16 | 32; };
template <> struct M64Form<16> { static constexpr int KB = 6, KE = 8, BLK = 16, V = 16 | 32; };
template <> struct M64Form<17> { static constexpr int KB = 7, KE = 9, BLK = 16, V = 16 | 32; };
// 18 and 21: the register budget.  Form 9 runs under a cap of kM64MaxReg
// registers per thread (16 resident warps per SM, a few bytes of spill in
// the setup); 18 is form 9 without the cap (8 warps), 21 groups of 9 / 11
// under the cap of 128.
constexpr int kM64MaxReg = 128;
template <> struct M64Form<18> : M64Form<9> {};
template <> struct M64Form<21> { static constexpr int KB = 9, KE = 11, BLK = 16, V = 16 | 32; };
// 42, 43: form 9 with smaller Euler groups, 10 squares (the default until
// lane chains) and 11; the default's 12 squares step tables of degree 24 and
// 22, no more registers than the 8-cube tables
template <> struct M64Form<42> { static constexpr int KB = 8, KE = 10, BLK = 16, V = 16 | 32; };
template <> struct M64Form<43> { static constexpr int KB = 8, KE = 11, BLK = 16, V = 16 | 32; };
// 49: the u form (flag 64): G0 = u^e from a table of u = prod (s+i) of degree
// K, groups of 12 cubes / 16 squares (tables of 13 + 34 and 17 + 31 entries,
// the default's register budget), with one REDC round per product of u^e
// (flag 128)
template <> struct M64Form<49> {
  static constexpr int KB = 12, KE = 16, BLK = 16, V = 16 | 32 | 64 | 128;
};

// a b 2^-64 mod p, below p + 2^12 for a, b < 2^38
__device__ __forceinline__ uint64_t m64_mm(uint64_t a, uint64_t b, const M64K &K) {
  uint32_t T0;
  uint64_t TY;
  m64_prod(a, b, T0, TY);
  return m64_redc2(T0, TY, K);
}
// v < 2p -> [0, p); canonical modular add and subtract
__device__ __forceinline__ uint64_t m64_once(uint64_t v, uint64_t p) { return v >= p ? v - p : v; }
__device__ __forceinline__ uint64_t m64_addm(uint64_t a, uint64_t b, uint64_t p) {
  return m64_once(a + b, p);
}
__device__ __forceinline__ uint64_t m64_subm(uint64_t a, uint64_t b, uint64_t p) {
  return a >= b ? a - b : a + p - b;
}

template <int ILP, bool CUBES, int AR, bool LANE = false>
__device__ __forceinline__ void tile_m64_grouped(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                                 int64_t &r0, int64_t &r1) {
  using F = M64Form<AR>;
  constexpr int V = F::V;
  constexpr int K = CUBES ? F::KB : F::KE;
  constexpr uint32_t BLK = F::BLK;
  constexpr int EX = CUBES ? 3 : 2;
  constexpr int DA = K * EX;
  constexpr int DB = (K - 1) * EX;
  // flag 64, the u form: G0 = u^EX with u = prod_{i<K} (s+i) from a table of
  // degree K (the rolled set-up only)
  constexpr bool UF = (V & 64) != 0;
  static_assert(!UF || ((V & 32) && !(V & 12)), "the u form needs the rolled set-up, plain adds");
  // flag 128: one 32-bit REDC round (a factor 2^-32) per product of u^EX
  // instead of two: u's value below 6p < 2^39.6 gives u u 2^-32 < 2^47.2 and
  // u^3 2^-64 < 2^55, still below 2^57, and every product of the pair
  // update stays below 2^96 (c0, c1 < p + 2^32 from the full rounds there)
  constexpr bool UH = (V & 128) != 0;
  static_assert(!UH || UF, "one-round products belong to the u form");
  constexpr int DT = UF ? K : DA;          // degree of the first table
  constexpr int DTOP = DT > DB ? DT : DB;  // set-up points 0 .. DTOP
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  M64K KK;
  KK.p = ctx.p;
  KK.p0 = (uint32_t)ctx.p;
  KK.p1 = (uint32_t)(ctx.p >> 32);
  KK.q = 0u - (uint32_t)ctx.q;  // -p^-1 mod 2^32
  KK.mhi = (uint32_t)((1ull << 62) / ctx.p);
  const uint32_t z32 = ctx.flags >> 16;                                // runtime zero
  const uint64_t np = 0ull - ctx.p;  // 2^64 - p, for the four-step shrink
  const uint32_t np0 = (uint32_t)np, np1 = (uint32_t)(np >> 32);
  constexpr int NF = (DA + DB) * M64Split<AR>::NFQ / 4;  // carry-chain entries
  const uint64_t nch = LANE ? ILP : 32 * ILP;  // lane chains: the lane owns the tile
  const uint64_t len = n / nch;
  const uint32_t rem = (uint32_t)(n - len * nch);
  const uint64_t G = len / K;
  uint64_t c0[ILP], c1[ILP], ga[ILP][DT + 1], gb[ILP][DB + 1];
  uint64_t s_tail[ILP];
  uint32_t n_tail[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) {
    const uint32_t ch = LANE ? k : k * 32 + lane;
    const uint64_t s = start + ch * len + (ch < rem ? ch : rem);
    const uint64_t L = len + (ch < rem ? 1 : 0);
    s_tail[k] = s + G * K;
    n_tail[k] = (uint32_t)(L - G * K);
    // Difference tables of the group polynomials at s, s + K, ..., s + DA K.
    // Each point's pair is built from the plain powers t = x^e of its K
    // consecutive x by the running recurrence P <- P t, Q <- Q t + P (start
    // P = t, Q = R) in the two-round REDC above, which gives
    // G0 = R^-(K-1) prod t_i and G1 = R^-(K-2) sum_i prod_{j != i} t_j: the
    // same factor R^-(K-1) on G0 and on R G1, so c1 / c0 is unchanged.  The
    // points are visited from the top down (x^e by backward differences) and
    // folded into the tables' diagonal as they come: e_j <- (-1)^j D^j.
    const uint64_t p = ctx.p;
    {
      uint64_t xr = s + (uint64_t)(K * (DTOP + 1) - 1);
      xr = xr >= p ? xr % p : xr;
      // the plain x of the current term (u form), kept as x + p: it falls by
      // at most K (DTOP + 1) < 2^10 during the set-up and stays positive
      uint64_t xc = xr + p;
      const uint64_t sq = (uint64_t)M.mulmod((int64_t)xr, (int64_t)xr);
      uint64_t t, d1, d2;
      if (EX == 3) {  // x^3, 3x^2 - 3x + 1, 6x - 6, 6
        t = (uint64_t)M.mulmod((int64_t)sq, (int64_t)xr);
        d1 = ((3 * sq + 1) % p + p - (3 * xr) % p) % p;
        d2 = (6 * xr + 6 * p - 6) % p;
      } else {        // x^2, 2x - 1, 2
        t = sq;
        d1 = (2 * xr + p - 1) % p;
        d2 = 2;
      }
      // one point: the pair (P, Q) of the K consecutive x from the current x
      // down, products not canonicalised (P, Pu < p + 2^12, Q < 2p + 2^13:
      // inputs below about 2^38 keep each product below p + 2^12); the
      // caller reduces them
      auto point = [&](uint64_t &P, uint64_t &Q, uint64_t &Pu) {
        P = 0;
        Q = ctx.one;
        Pu = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          if (i == 0) {
            P = t;
            if (UF) Pu = xc;
          } else {
            Q = m64_mm(Q, t, KK) + P;
            P = m64_mm(P, t, KK);
            if (UF) Pu = m64_mm(Pu, xc, KK);
          }
          t = m64_subm(t, d1, p);
          d1 = m64_subm(d1, d2, p);
          if (EX == 3) d2 = m64_subm(d2, 6, p);
          if (UF) xc -= 1;
        }
        Q = m64_once(m64_once(Q, p), p);
      };
      if constexpr ((V & 32) != 0) {
        // the point loop rolled (flag 32): a few hundred instructions of code
        // instead of DA + 1 unrolled copies; the table indices stay
        // compile-time, and each point folds into the diagonals over their
        // whole length (with zeros before the first point, a difference of
        // order j <= D at the last point involves only its last j + 1 points)
#pragma unroll
        for (int j = 0; j <= DT; ++j) ga[k][j] = 0;
#pragma unroll
        for (int j = 0; j <= DB; ++j) gb[k][j] = 0;
#pragma unroll 1
        for (int m = DTOP; m >= 0; --m) {
          uint64_t P, Q, Pu;
          point(P, Q, Pu);
          uint64_t nv;
          if (m <= DT) {
            nv = m64_once(UF ? Pu : P, p);
#pragma unroll
            for (int j = 0; j <= DT; ++j) {
              const uint64_t old = ga[k][j];
              ga[k][j] = nv;
              if (j < DT) nv = m64_subm(nv, old, p);
            }
          }
          if (m <= DB) {
            nv = Q;
#pragma unroll
            for (int j = 0; j <= DB; ++j) {
              const uint64_t old = gb[k][j];
              gb[k][j] = nv;
              if (j < DB) nv = m64_subm(nv, old, p);
            }
          }
        }
      } else {
#pragma unroll
        for (int m = DA; m >= 0; --m) {
          uint64_t P, Q, Pu;
          point(P, Q, Pu);
          // fold the new point into the diagonals (point DA - m of the sequence)
          uint64_t nv = m64_once(P, p);
#pragma unroll
          for (int j = 0; j <= DA - m; ++j) {
            const uint64_t old = ga[k][j];
            ga[k][j] = nv;
            if (j < DA - m) nv = m64_subm(nv, old, p);
          }
          if (m <= DB) {
            nv = Q;
#pragma unroll
            for (int j = 0; j <= DB - m; ++j) {
              const uint64_t old = gb[k][j];
              gb[k][j] = nv;
              if (j < DB - m) nv = m64_subm(nv, old, p);
            }
          }
        }
      }
#pragma unroll
      for (int j = 1; j <= DT; j += 2) ga[k][j] = ga[k][j] ? p - ga[k][j] : 0;
#pragma unroll
      for (int j = 1; j <= DB; j += 2) gb[k][j] = gb[k][j] ? p - gb[k][j] : 0;
    }
    c0[k] = ctx.one;
    c1[k] = 0;
  }
  for (uint64_t g = 0; g < G;) {
    const uint32_t nb = (G - g < BLK) ? (uint32_t)(G - g) : BLK;
#pragma unroll 1
    for (uint32_t r = 0; r < nb; ++r) {
#pragma unroll
      for (int k = 0; k < ILP; ++k) {
        uint32_t T0;
        uint64_t TY;
        uint64_t A = ga[k][0];
        if constexpr (UF) {
          // G0 = u^EX: u's value brought below 6p < 2^40 (both factors of a
          // product below 2^40 keep it under 2^80), then EX - 1 products
          const uint64_t Us = m64_shrink_q(A, KK, np0, np1);
          m64_prod(Us, Us, T0, TY);
          A = UH ? m64_redc1(T0, TY, KK) : m64_redc2(T0, TY, KK);  // < 2^47.2 or p + 2^16
          if (EX == 3) {
            m64_prod(A, Us, T0, TY);
            A = UH ? m64_redc1(T0, TY, KK) : m64_redc2(T0, TY, KK);  // < 2^55 or p + 2^16
          }
        }
        m64_prod(c0[k], A, T0, TY);
        const uint64_t n0 = m64_redc2(T0, TY, KK);
        m64_prod2(c1[k], A, c0[k], gb[k][0], T0, TY);
        c1[k] = m64_redc2(T0, TY, KK);
        c0[k] = n0;
#pragma unroll
        for (int j = 0; j < DT; ++j) {
          if ((V & 12) && j < NF) {
            if (V & 8) add64_cc_z(ga[k][j], ga[k][j + 1], z32);
            else add64_cc(ga[k][j], ga[k][j + 1]);
          } else {
            ga[k][j] = ga[k][j] + ga[k][j + 1];
          }
        }
#pragma unroll
        for (int j = 0; j < DB; ++j) {
          if ((V & 12) && DA + j < NF) {
            if (V & 8) add64_cc_z(gb[k][j], gb[k][j + 1], z32);
            else add64_cc(gb[k][j], gb[k][j + 1]);
          } else {
            gb[k][j] = gb[k][j] + gb[k][j + 1];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
#pragma unroll
      for (int j = 0; j < DT; ++j)
        ga[k][j] = (V & 16) ? m64_shrink_q(ga[k][j], KK, np0, np1) : m64_shrink(ga[k][j], KK);
#pragma unroll
      for (int j = 0; j < DB; ++j)
        gb[k][j] = (V & 16) ? m64_shrink_q(gb[k][j], KK, np0, np1) : m64_shrink(gb[k][j], KK);
    }
    g += nb;
  }
  if constexpr (UF) {
    // u^EX carries R^-(EX-1)K more than the pair tables' G0 (with one-round
    // products R^-(EX-1)(K-1/2), R = 2^64): scale c1 back once by that
    // factor, as f = R^(1-(EX-1)K) (or the like) times R^-1 in the product
    uint64_t f = ctx.one;
    if constexpr (UH) {
#pragma unroll 1
      for (int i = 0; i < (EX - 1) * (2 * K - 1); ++i) f = m64_redc1(ulo(f), uhi(f), KK);
    } else {
#pragma unroll 1
      for (int i = 0; i < (EX - 1) * K; ++i) f = m64_mm(f, 1, KK);
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) c1[k] = m64_mm(c1[k], f, KK);
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
  if (!LANE) warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// ------------------------------------------------------------------ accumulate
// One warp tile g of plan P: find its (prime, row) segment, sum its range of
// terms, merge the lanes, and store the tile's (c0, c1) pair.
// ---- the paper's own arithmetic, kept as an ablation (arith 23) -------------
// Sec. 3 ("Method for primes p < 6e10" and its improvements 1-2): plain
// residues; a product mod p of a = a0 + a1 2^32 and b = b0 + b1 2^32 by
// eqn 3.15, ab = a0 b0 + a1 b0 2^32 + b1 (a0 2^32 + a1 2^64), each piece a
// native 64-bit product reduced by a remainder whose quotient comes from a
// double-precision product with 1/p (exact after at most two corrections
// each way, as every reduced value is below 2^64 and p >= 2^11); for p < 2^32
// one native product and one such remainder.  Terms s^e by forward
// differences (improvement 1), single eqn 3.12 steps.
__device__ __forceinline__ uint64_t rem_fp64(uint64_t x, uint64_t p, double pinv) {
  const uint64_t q = (uint64_t)((double)x * pinv);
  int64_t r = (int64_t)(x - q * p);
  const int64_t sp = (int64_t)p;
  if (r < 0) r += sp;
  if (r < 0) r += sp;
  if (r >= sp) r -= sp;
  if (r >= sp) r -= sp;
  return (uint64_t)r;
}

__device__ __forceinline__ uint64_t mulmod_split(uint64_t a, uint64_t b, uint64_t p, double pinv,
                                                 uint64_t r64) {
  if (p < (1ull << 32)) return rem_fp64(a * b, p, pinv);
  const uint64_t a0 = a & 0xffffffffull, a1 = a >> 32, b0 = b & 0xffffffffull, b1 = b >> 32;
  const uint64_t t0 = rem_fp64(a0 * b0, p, pinv);
  // a1 b0 2^32: a1 b0 < 2^37, reduced, then the shift in two steps of 27 and 5 bits
  uint64_t t1 = rem_fp64(a1 * b0, p, pinv);
  t1 = rem_fp64(rem_fp64(t1 << 27, p, pinv) << 5, p, pinv);
  // b1 (a0 2^32 + a1 2^64): both inside the bracket reduced, 2^64 mod p precomputed
  const uint64_t u = rem_fp64(a0 << 32, p, pinv) + a1 * r64;
  const uint64_t t2 = rem_fp64(b1 * u, p, pinv);
  return rem_fp64(t0 + t1 + t2, p, pinv);
}

template <bool CUBES>
__device__ __forceinline__ void tile_paper(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                           int64_t &r0, int64_t &r1) {
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  const uint64_t p = ctx.p;
  const double pinv = 1.0 / (double)p;
  // 2^64 mod p, needed for p >= 2^32 only, where R = 2^64 and ctx.one = R mod p
  const uint64_t r64 = (ctx.flags & 1u) ? ctx.one : 0;
  const uint64_t len = n / 32, rem = n - len * 32;
  const uint64_t s = start + lane * len + (lane < rem ? lane : rem);
  const uint64_t L = len + (lane < rem ? 1 : 0);
  // s^e and its forward differences, canonical in [0, p)
  const uint64_t sq = mulmod_split(s, s, p, pinv, r64);
  uint64_t t, d1, d2;
  if (CUBES) {
    t = mulmod_split(sq, s, p, pinv, r64);
    d1 = rem_fp64(3 * sq + 3 * s + 1, p, pinv);
    d2 = rem_fp64(6 * s + 6, p, pinv);
  } else {
    t = sq;
    d1 = rem_fp64(2 * s + 1, p, pinv);
    d2 = 2;
  }
  const uint64_t d3 = CUBES ? 6 : 0;
  uint64_t c0 = 1, c1 = 0;
  for (uint64_t i = 0; i < L; ++i) {
    c1 = mulmod_split(c1, t, p, pinv, r64) + c0;  // eqn 3.12
    c1 = c1 >= p ? c1 - p : c1;
    c0 = mulmod_split(c0, t, p, pinv, r64);
    t += d1;
    t = t >= p ? t - p : t;
    d1 += d2;
    d1 = d1 >= p ? d1 - p : d1;
    if (CUBES) {
      d2 += d3;
      d2 = d2 >= p ? d2 - p : d2;
    }
  }
  // c1 / c0 = S; the merge and the finaliser expect R S: scale c1 by R mod p
  c1 = mulmod_split(c1, ctx.one, p, pinv, r64);
  int64_t a0 = (int64_t)c0, a1 = (int64_t)c1;
  warp_merge(M, a0, a1);
  r0 = a0;
  r1 = a1;
}

// ---- general index (arith 24): sums of s^-e for any 2 <= e <= 16 ----------
// Single eqn 3.12 steps on canonical Montgomery values (the generic Mont
// arithmetic of either path), terms s^e from a forward-difference table of
// degree e.
constexpr int kGenEMax = 16;
__device__ __forceinline__ void tile_general(const PrimeCtx &ctx, uint64_t start, uint64_t n,
                                             uint32_t e, int64_t &r0, int64_t &r1) {
  const int lane = threadIdx.x & 31;
  const Mont M(ctx);
  const uint64_t len = n / 32, rem = n - len * 32;
  const uint64_t s = start + lane * len + (lane < rem ? lane : rem);
  const uint64_t L = len + (lane < rem ? 1 : 0);
  int64_t d[kGenEMax + 1];
#pragma unroll
  for (int i = 0; i <= kGenEMax; ++i) {
    d[i] = 0;
    if ((uint32_t)i <= e) {
      uint64_t x = s + (uint64_t)i;
      if (x >= ctx.p) x -= ctx.p;
      d[i] = M.from_mont(M.pow(M.to_mont((int64_t)x), e));  // x^e mod p, plain
    }
  }
#pragma unroll
  for (int j = 1; j <= kGenEMax; ++j)
#pragma unroll
    for (int i = kGenEMax; i >= j; --i)
      if ((uint32_t)i <= e) d[i] = M.sub(d[i], d[i - 1]);
  int64_t c0 = M.one, c1 = 0;
  for (uint64_t it = 0; it < L; ++it) {
    const int64_t t = d[0];
    c1 = M.add(M.mul(c1, t), c0);  // REDC(c1 t) + c0: c1 / c0 grows by R / t
    c0 = M.mul(c0, t);
#pragma unroll
    for (int j = 0; j < kGenEMax; ++j)
      if ((uint32_t)j < e) d[j] = M.add(d[j], d[j + 1]);
  }
  warp_merge(M, c0, c1);
  r0 = c0;
  r1 = c1;
}

// Group sizes (KC cubes, KS squares; 0: 2 cubes, 3 squares) and ALU-only
// table additions per group (NFC of a Bernoulli group's, NFS of an Euler
// group's) of each grouped 32-bit formulation.  9: 4 of 9 and 2 of 10 (the
// fastest on GB300 of 0, 2..6 and all); 25: none, 26: 4 and 4, 27: 6 and 6,
// 28: all (ablation).  29..31 are 9 with larger groups: 3 cubes (15
// additions, 6 ALU-only), 4 squares (14 additions, 4 ALU-only), or both (31,
// the default with warp tiles).  39: larger groups still, 4 cubes / 5 squares
// (21 and 18 additions, 6 and 4 ALU-only); of 4 / 5 with 8 / 6 ALU-only,
// 3 / 5 and 4 / 4 it was the fastest, and faster than 31 on long sums: with
// lane chains (where every chain is long) it is the default, at ILP 1.
template <int AR> struct M31Form { static constexpr int KC = 0, KS = 0, NFC = 4, NFS = 2; };
template <> struct M31Form<25> { static constexpr int KC = 0, KS = 0, NFC = 0, NFS = 0; };
template <> struct M31Form<26> { static constexpr int KC = 0, KS = 0, NFC = 4, NFS = 4; };
template <> struct M31Form<27> { static constexpr int KC = 0, KS = 0, NFC = 6, NFS = 6; };
template <> struct M31Form<28> { static constexpr int KC = 0, KS = 0, NFC = 10, NFS = 10; };
template <> struct M31Form<29> { static constexpr int KC = 3, KS = 0, NFC = 6, NFS = 2; };
template <> struct M31Form<30> { static constexpr int KC = 0, KS = 4, NFC = 4, NFS = 4; };
template <> struct M31Form<31> { static constexpr int KC = 3, KS = 4, NFC = 6, NFS = 4; };
template <> struct M31Form<39> { static constexpr int KC = 4, KS = 5, NFC = 6, NFS = 4; };
// 40, 41, 44: larger groups still, for lane chains (every chain long): 5
// cubes / 6 squares (27 and 22 additions, 8 and 5 ALU-only), 4 cubes / 6
// squares (41, the default with lane chains), 4 cubes / 7 squares
template <> struct M31Form<40> { static constexpr int KC = 5, KS = 6, NFC = 8, NFS = 5; };
template <> struct M31Form<41> { static constexpr int KC = 4, KS = 6, NFC = 6, NFS = 5; };
template <> struct M31Form<44> { static constexpr int KC = 4, KS = 7, NFC = 6, NFS = 6; };
// 45..47: the u form (tile_m31_grouped, UF): G0 = u^e from a table of
// u = prod (s+i) of degree K, so a group steps K + e(K-1) table entries
// instead of 2eK - e, for e - 1 more products per group; groups of 8 cubes
// / 10 squares (45), 6 / 8 (46) and 10 / 12 (47)
template <int AR> struct M31UF { static constexpr bool on = false; };
template <> struct M31UF<45> { static constexpr bool on = true; };
template <> struct M31UF<46> { static constexpr bool on = true; };
template <> struct M31UF<47> { static constexpr bool on = true; };
template <> struct M31UF<51> { static constexpr bool on = true; };
template <> struct M31UF<52> { static constexpr bool on = true; };
template <> struct M31Form<45> { static constexpr int KC = 8, KS = 10, NFC = 8, NFS = 8; };
template <> struct M31Form<46> { static constexpr int KC = 6, KS = 8, NFC = 6, NFS = 6; };
template <> struct M31Form<47> { static constexpr int KC = 10, KS = 12, NFC = 10, NFS = 10; };
// 51, 52: form 45 with more (12 / 10) and fewer (4 / 4) of a group's table
// additions as ALU-only three-input adds
template <> struct M31Form<51> { static constexpr int KC = 8, KS = 10, NFC = 12, NFS = 10; };
template <> struct M31Form<52> { static constexpr int KC = 8, KS = 10, NFC = 4, NFS = 4; };
// 48 (lane chains): per warp, the u form of 45 for pieces of at least
// Plan::uform_min[0] terms (3072 by default: its set-up visits e(K-1) + 1
// points of K terms, about three times form 41's, and pays on long pieces
// only) and form 41 below
template <> struct M31Form<48> : M31Form<41> {};
template <> struct M31Form<49> : M31Form<41> {};  // 49, 50: 48 on the 32-bit kernel
template <> struct M31Form<50> : M31Form<41> {};
// 64-bit path, form 50: per warp the u form of 49 on pieces of at least
// Plan::uform_min[1] terms (32768 by default: its set-up visits 34 points of
// 12 terms), form 9 below

template <bool WIDE, int ILP, int AR, bool LANE = false>
__device__ __forceinline__ void process_tile(const Plan &P, uint32_t g) {
  const int lane = threadIdx.x & 31;
  bool live = true;
  uint32_t slot, j;
  uint64_t start, n;
  if constexpr (LANE) {
    // g is a warp of lane chains: this lane's piece from the sorted list; a
    // padding lane repeats lane 0's piece (same code path, nothing stored)
    const PieceRec *rp = P.rec + 32 * (size_t)g + lane;
    uint64_t st = __ldg(&rp->start);
    uint32_t nn = __ldg(&rp->n), t = __ldg(&rp->tile), sl = __ldg(&rp->slot), rw = __ldg(&rp->row);
    live = t != kNoChain;
    const uint64_t st0 = __shfl_sync(0xffffffffu, st, 0);
    const uint32_t nn0 = __shfl_sync(0xffffffffu, nn, 0), t0 = __shfl_sync(0xffffffffu, t, 0);
    const uint32_t sl0 = __shfl_sync(0xffffffffu, sl, 0), rw0 = __shfl_sync(0xffffffffu, rw, 0);
    g = live ? t : t0;
    start = live ? st : st0;
    n = live ? nn : nn0;
    slot = live ? sl : sl0;
    j = live ? rw : rw0;
  } else {
    // segment owning tile g (the planner's tile -> segment map)
    const uint32_t s = __ldg(&P.tile_seg[g]);
    slot = s / P.rows_pp;
    j = s - slot * P.rows_pp;
    const uint32_t k = g - P.seg_first[s], T = P.seg_tiles[s];
    const uint64_t cnt = P.seg_cnt[s];
    const uint64_t b0 = cnt * k / T, b1 = cnt * (k + 1) / T;
    start = P.seg_lo[s] + b0;
    n = b1 - b0;
  }
  const PrimeCtx ctx = P.ctx[slot];
  int64_t r0, r1;
  // single-term form used beside the grouped one
  constexpr int AS = (AR == 5 || AR >= 8) ? 4 : AR;
  // group sizes and ALU-only table additions of the grouped 32-bit form
  constexpr int NFC = M31Form<AR>::NFC, NFS = M31Form<AR>::NFS;
  constexpr int KC = M31Form<AR>::KC, KS = M31Form<AR>::KS;
  constexpr bool UFM = M31UF<AR>::on;
  const bool grp_ok = n >= (LANE ? 1ull : 32ull) * ILP * kGroupMinChain;
  // forms 48..50: the warp's pieces are sorted by length, so lane 0's decides
  constexpr bool ADAPT = AR >= 48 && AR <= 50;
  bool ufw = false;
  if constexpr (ADAPT && !WIDE) ufw = __shfl_sync(0xffffffffu, n, 0) >= P.uform_min[0];
  if constexpr (AR == 50 && WIDE) ufw = __shfl_sync(0xffffffffu, n, 0) >= P.uform_min[1];
  using F45 = M31Form<45>;
  if (AR == 24) {
    tile_general(ctx, start, n, j < P.rows_b ? P.gen_e_b : P.gen_e_e, r0, r1);
  } else if (AR == 23) {
    if (j < P.rows_b) tile_paper<true>(ctx, start, n, r0, r1);
    else tile_paper<false>(ctx, start, n, r0, r1);
  } else if (!WIDE && (ctx.flags & 1u)) {
    // 2^30 <= p < 2^31 on the 32-bit kernel: the unsigned grouped form with
    // this formulation's group sizes, single 64-bit terms on short tiles
    if (ADAPT && ufw && grp_ok) {
      if (j < P.rows_b) tile_m31_grouped<ILP, true, 7, F45::NFC, F45::KC, true, LANE, true>(ctx, start, n, r0, r1);
      else tile_m31_grouped<ILP, false, 7, F45::NFS, F45::KS, true, LANE, true>(ctx, start, n, r0, r1);
    } else if (AR >= 9 && grp_ok) {
      if (j < P.rows_b) tile_m31_grouped<ILP, true, 7, NFC, KC, true, LANE, UFM>(ctx, start, n, r0, r1);
      else tile_m31_grouped<ILP, false, 7, NFS, KS, true, LANE, UFM>(ctx, start, n, r0, r1);
    } else {
      if (j < P.rows_b) tile_m64<ILP, true, LANE>(ctx, start, n, r0, r1);
      else tile_m64<ILP, false, LANE>(ctx, start, n, r0, r1);
    }
  } else if (!WIDE && AR == 5 && grp_ok) {
    if (j < P.rows_b) tile_m31_grouped<ILP, true, 5>(ctx, start, n, r0, r1);
    else tile_m31_grouped<ILP, false, 5>(ctx, start, n, r0, r1);
  } else if (!WIDE && ADAPT && ufw && grp_ok) {
    if (j < P.rows_b) tile_m31_grouped<ILP, true, 7, F45::NFC, F45::KC, false, LANE, true>(ctx, start, n, r0, r1);
    else tile_m31_grouped<ILP, false, 7, F45::NFS, F45::KS, false, LANE, true>(ctx, start, n, r0, r1);
  } else if (!WIDE && AR >= 7 && grp_ok && j >= P.rows_b) {
    tile_m31_grouped<ILP, false, 7, NFS, KS, false, LANE, UFM>(ctx, start, n, r0, r1);
  } else if (!WIDE && AR >= 9 && grp_ok) {
    tile_m31_grouped<ILP, true, 7, NFC, KC, false, LANE, UFM>(ctx, start, n, r0, r1);
  } else if (!WIDE) {
    if (j < P.rows_b) tile_m31<ILP, true, AS, LANE>(ctx, start, n, r0, r1);
    else tile_m31<ILP, false, AS, LANE>(ctx, start, n, r0, r1);
  } else if (AR == 50 && grp_ok) {  // 64-bit: the u form on long pieces
    if (ufw) {
      if (j < P.rows_b) tile_m64_grouped<ILP, true, 49, LANE>(ctx, start, n, r0, r1);
      else tile_m64_grouped<ILP, false, 49, LANE>(ctx, start, n, r0, r1);
    } else {
      if (j < P.rows_b) tile_m64_grouped<ILP, true, 9, LANE>(ctx, start, n, r0, r1);
      else tile_m64_grouped<ILP, false, 9, LANE>(ctx, start, n, r0, r1);
    }
  } else if (AR >= 9 && grp_ok) {
    if (j < P.rows_b) tile_m64_grouped<ILP, true, AR, LANE>(ctx, start, n, r0, r1);
    else tile_m64_grouped<ILP, false, AR, LANE>(ctx, start, n, r0, r1);
  } else {
    if (j < P.rows_b) tile_m64<ILP, true, LANE>(ctx, start, n, r0, r1);
    else tile_m64<ILP, false, LANE>(ctx, start, n, r0, r1);
  }
  if (LANE ? live : lane == 0)
    P.partials[g] = make_ulonglong2((unsigned long long)r0, (unsigned long long)r1);
}

template <bool WIDE, int ILP, int AR, bool LANE = false>
__device__ __forceinline__ void accumulate_loop(const Plan &P) {
  const int lane = threadIdx.x & 31;
  if constexpr (LANE) {
    // warps of lane chains, [0, lane_w[0]) on the 32-bit kernel and
    // [lane_w[0], lane_w[1]) on the 64-bit one, taken from the top (longest
    // chains of each class first)
    const uint32_t w0 = WIDE ? P.lane_w[0] : 0u, w1 = WIDE ? P.lane_w[1] : P.lane_w[0];
    uint32_t *counter = P.counters + (WIDE ? 1 : 0);
    for (;;) {
      uint32_t g = 0;
      if (lane == 0) g = atomicAdd(counter, 1u);
      g = __shfl_sync(0xffffffffu, g, 0);
      if (g >= w1 - w0) break;
      process_tile<WIDE, ILP, AR, true>(P, w1 - 1 - g);
    }
    return;
  }
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

// At least 3 resident blocks of 256 threads per SM: a register budget of up
// to 85 per thread.  Without the minimum the compiler fits the 32-bit
// grouped kernel into 64 registers (4 blocks) and schedules its group loop
// tighter, which measured slower on GB300 than 3 blocks of 70 registers.
template <bool WIDE, int ILP, int AR, bool LANE = false>
__global__ void __launch_bounds__(kAccThreads, 3) k_accumulate(Plan P) {
  accumulate_loop<WIDE, ILP, AR, LANE>(P);
}

// The 64-bit path with a register cap (any block size): fewer registers per
// thread, more resident warps.
template <int AR, int MAXREG, bool LANE = false>
__global__ void __maxnreg__(MAXREG) k_accumulate_m64cap(Plan P) {
  accumulate_loop<true, 1, AR, LANE>(P);
}

// Epoch form: tiles of several plans (one per request of a serving loop),
// given as items {plan, first tile, count, prefix}; the items' tiles are
// taken from one counter, each item from its top tile down.  LANE: the plans
// hold lane chains and a "tile" is a warp of their sorted tile list.
template <bool WIDE, int ILP, int AR, bool LANE = false>
__global__ void __maxnreg__(kM64MaxReg)
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
    process_tile<WIDE, ILP, AR, LANE>(plans[it.plan], it.first + it.count - 1 - (g - it.prefix));
  }
}

// Epoch form with both arithmetic paths in one launch: items with bit 31 of
// `plan` set are 64-bit-path tiles.  One launch (and one tail) per epoch.
template <int I31, int I64, bool LANE = false>
__global__ void __maxnreg__(kM64MaxReg)
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
    if (it.plan >> 31) process_tile<true, I64, LANE ? 50 : 9, LANE>(plans[it.plan & 0x7fffffffu], tile);
    else process_tile<false, I31, 48, LANE>(plans[it.plan], tile);
  }
}

// Non-persistent epoch form: one warp per tile (grid = the epoch's tiles in
// one-warp blocks), so warps retire tile by tile and the block scheduler
// hands their slots to whatever is pending -- the next epoch, or admission
// kernels on a higher-priority stream -- without a persistent grid's tail.
template <int I31, int I64, bool LANE = false>
__global__ void __maxnreg__(kM64MaxReg)
    k_epoch_tiles(const EpochItem *items, uint32_t n_items, uint32_t total, const Plan *plans) {
  const uint32_t g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= total) return;
  uint32_t lo = 0, hi = n_items;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&items[mid].prefix) <= g) lo = mid; else hi = mid;
  }
  const EpochItem it = items[lo];
  const uint32_t tile = it.first + it.count - 1 - (g - it.prefix);
  if (it.plan >> 31) process_tile<true, I64, LANE ? 50 : 9, LANE>(plans[it.plan & 0x7fffffffu], tile);
  else process_tile<false, I31, 48, LANE>(plans[it.plan], tile);
}

// ------------------------------------------------------------------ getters
using AccKernel = void (*)(Plan);
using EpochKernel = void (*)(const EpochItem *, uint32_t, uint32_t, const Plan *, uint32_t *);
// 32-bit path: formulation 1..9, ILP 1, 2 (any formulation) or 4 (formulation 9)
AccKernel acc_kernel_m31(int arith, int ilp);
// 64-bit path: formulation 1 (single terms, ILP 1, 2 or 4) or 9 (grouped
// default, one chain per thread)
AccKernel acc_kernel_m64(int arith, int ilp);
// 64-bit path formulations kept for ablation (arith 10..22), one chain per thread
AccKernel acc_kernel_m64x(int arith, int ilp);
// forms 16..18, 19..21 and 22..24, each its own translation unit
// (acc_kernel_m64x falls through to y, y to z, z to w)
AccKernel acc_kernel_m64y(int arith, int ilp);
AccKernel acc_kernel_m64z(int arith, int ilp);
AccKernel acc_kernel_m64w(int arith, int ilp);
AccKernel acc_kernel_m64v(int arith, int ilp);  // forms 32..36 (w falls through to v)
// 32-bit path: formulation 9 with other ALU-only splits or group sizes (arith 25..31), ILP 1 or 2
AccKernel acc_kernel_m31x(int arith, int ilp);
// lane chains: the 32-bit grouped formulations 39 (default) and 31, ILP 1 or
// 2, and the 64-bit grouped default (one chain per thread)
AccKernel acc_kernel_lane31(int arith, int ilp);
AccKernel acc_kernel_lane64(int arith);
// lane-chain forms 40, 41 (the default), 44 (32-bit groups) and 42, 43
// (64-bit groups)
AccKernel acc_kernel_lane31x(int arith, int ilp);
AccKernel acc_kernel_lane31u(int arith, int ilp);  // the u form, 45..48
AccKernel acc_kernel_lane64u(int arith);            // the 64-bit u form, 49, 50
AccKernel acc_kernel_lane64x(int arith);
AccKernel acc_kernel_m31y(int arith, int ilp);  // form 39 (x falls through to y)
// serving-loop epoch kernels (the default formulations: 31 on the 32-bit path,
// 9 with one chain per thread on the 64-bit path)
EpochKernel epoch_kernel(bool wide, int ilp, bool lane);
EpochKernel epoch_mixed_kernel(int ilp31, int ilp64, bool lane);
using EpochTilesKernel = void (*)(const EpochItem *, uint32_t, uint32_t, const Plan *);
EpochTilesKernel epoch_tiles_kernel(int ilp31, bool lane);

}  // namespace wv
