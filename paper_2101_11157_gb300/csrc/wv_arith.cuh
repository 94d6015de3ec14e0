// wv_arith.cuh -- exact modular arithmetic for the residue kernels.
//
// All arithmetic is integer and exact.  Two Montgomery representations:
//
//  * M31: p < 2^30, R = 2^32, values held as SIGNED 32-bit integers.
//    redc(a, b) = (a b - m p) / 2^32 with m = (a b) p^-1 mod 2^32 taken as a
//    signed 32-bit value; the low words of a b and m p agree, so the result
//    is exactly hi32(a b) - hi32(m p).  For |a| < 2p, |b| <= p it satisfies
//    |redc| < (2p^2 + 2^31 p) / 2^32 < p: no correction step is needed, and
//    the accumulation of eqn 3.12 keeps c0 in (-p, p) and c1 in (-2p, 2p).
//  * M64: p < 2^37, R = 2^64, the same construction on signed 64-bit values
//    (hi64 via __mul64hi).
//
// The hot loop multiplies a Montgomery-form accumulator by a PLAIN term t:
// redc(c R, t) = c t R (mod p), so t = s^3 or s^2 never needs converting.
// With tq = t p^-1 (one multiply per term) the two products c0 t and c1 t
// share it: m = c tq = (c t) p^-1 mod R.
#pragma once
#include <stdint.h>

namespace wv {

// ---------------------------------------------------------------- context
struct PrimeCtx {
  uint64_t p;     // the prime
  uint64_t q;     // p^-1 mod 2^64 (low 32 bits = p^-1 mod 2^32)
  uint64_t one;   // R mod p (Montgomery form of 1), canonical
  uint64_t r2;    // R^2 mod p, canonical
  uint32_t orig;  // index of this prime in the caller's array
  uint32_t flags; // bit0: wide (M64) path; bit1: special/invalid (no sums)
};

constexpr uint64_t kM31Limit = 1ull << 30;
constexpr uint64_t kPMax = 1ull << 37;

// floor(n p / d) for n <= d < 2^32 and p < 2^64, in 64-bit words: with
// p = a d + b, n p / d = n a + n b / d, where n a <= n p / d < 2^64 and
// n b < 2^64.  The planner uses it for the endpoints x p, y p of every sum.
__host__ __device__ inline uint64_t floor_frac_times(uint32_t n, uint32_t d, uint64_t p) {
  const uint64_t a = p / d, b = p % d;
  return (uint64_t)n * a + ((uint64_t)n * b) / d;
}

__host__ __device__ inline uint64_t inv_mod_2_64(uint64_t p) {
  uint64_t x = p;  // correct to 3 bits for odd p
  for (int i = 0; i < 5; ++i) x *= 2 - p * x;
  return x;
}

// 2^k mod p by doubling (p < 2^62), exact with 64-bit words.
__host__ __device__ inline uint64_t pow2_mod(unsigned k, uint64_t p) {
  uint64_t r = 1 % p;
  for (unsigned i = 0; i < k; ++i) {
    r <<= 1;
    if (r >= p) r -= p;
  }
  return r;
}
// x * 2^k mod p by doubling, x < p < 2^62
__host__ __device__ inline uint64_t shl_mod(uint64_t x, unsigned k, uint64_t p) {
  for (unsigned i = 0; i < k; ++i) {
    x <<= 1;
    if (x >= p) x -= p;
  }
  return x;
}

__host__ __device__ inline PrimeCtx make_ctx(uint64_t p, uint32_t orig) {
  PrimeCtx c;
  c.p = p;
  c.orig = orig;
  c.flags = 0;
  c.q = inv_mod_2_64(p);
  if (p < kM31Limit) {
    c.one = pow2_mod(32, p);
    c.r2 = shl_mod(c.one, 32, p);
  } else {
    c.flags |= 1u;
    c.one = pow2_mod(64, p);
    c.r2 = shl_mod(c.one, 64, p);
  }
  return c;
}

// ---------------------------------------------------------------- wide products
// a * b as a 64-bit product, and a * b + c with a 64-bit addend, each one
// instruction (PTX mul.wide / mad.wide).
__device__ __forceinline__ int64_t mul_wide(int32_t a, int32_t b) {
  int64_t d;
  asm("mul.wide.s32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ int64_t mad_wide(int32_t a, int32_t b, int64_t c) {
  int64_t d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
// high word of a 64-bit value (no instruction: the upper register of the pair)
__device__ __forceinline__ int32_t hi32(int64_t v) {
  int32_t hi;
  asm("{\n\t.reg .b32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=r"(hi) : "l"(v));
  return hi;
}
__device__ __forceinline__ int32_t lo32(int64_t v) {
  int32_t lo;
  asm("{\n\t.reg .b32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=r"(lo) : "l"(v));
  return lo;
}
// the 64-bit value with high word h and low word 0
__device__ __forceinline__ int64_t hi_word(int32_t h) {
  int64_t v;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "r"(0), "r"(h));
  return v;
}

// ---------------------------------------------------------------- M31
__device__ __forceinline__ int32_t m31_redc(int32_t a, int32_t b, int32_t p, uint32_t q) {
  int32_t hi = __mulhi(a, b);
  uint32_t lo = (uint32_t)a * (uint32_t)b;
  int32_t m = (int32_t)(lo * q);
  return hi - __mulhi(m, p);
}
// x in (-2p, 2p) -> [0, p)
__device__ __forceinline__ int32_t m31_canon(int32_t x, int32_t p) {
  x += (x >> 31) & p;
  x += (x >> 31) & p;
  return (x >= p) ? x - p : x;
}
__device__ __forceinline__ int32_t m31_add(int32_t a, int32_t b, int32_t p) {  // canonical in/out
  int32_t x = a + b;
  return (x >= p) ? x - p : x;
}
// canonical Montgomery product
__device__ __forceinline__ int32_t m31_mul(int32_t a, int32_t b, int32_t p, uint32_t q) {
  return m31_canon(m31_redc(a, b, p, q), p);
}

// Branch-free p < 2^30 residue arithmetic for per-chain set-up: canonical
// values in [0, p) as unsigned words; add and subtract by the unsigned
// minimum of the two candidates (the wrapped one is the larger).
struct M31Set {
  int32_t p;
  uint32_t q;
  uint32_t one, r2, c1, c2, c6;  // R, R^2 mod p; the plain constants 1, 2, 6 mod p
  __device__ __forceinline__ explicit M31Set(const PrimeCtx &c)
      : p((int32_t)c.p), q((uint32_t)c.q), one((uint32_t)c.one), r2((uint32_t)c.r2),
        c1(c.p > 1 ? 1u : 0u), c2(c.p > 2 ? 2u : (uint32_t)(2 % c.p)),
        c6(c.p > 6 ? 6u : (uint32_t)(6 % c.p)) {}
  __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const {  // a b R^-1
    return (uint32_t)m31_mul((int32_t)a, (int32_t)b, p, q);
  }
  __device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b) const {  // a b
    return mul(mul(a, b), r2);
  }
  __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) const {
    const uint32_t x = a + b;
    return min(x, x - (uint32_t)p);
  }
  __device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b) const {
    const uint32_t x = a - b;
    return min(x, x + (uint32_t)p);
  }
};

// ---------------------------------------------------------------- M64
__device__ __forceinline__ int64_t m64_redc(int64_t a, int64_t b, int64_t p, uint64_t q) {
  int64_t hi = __mul64hi(a, b);
  uint64_t lo = (uint64_t)a * (uint64_t)b;
  int64_t m = (int64_t)(lo * q);
  return hi - __mul64hi(m, p);
}
__device__ __forceinline__ int64_t m64_canon(int64_t x, int64_t p) {
  x += (x >> 63) & p;
  x += (x >> 63) & p;
  return (x >= p) ? x - p : x;
}
__device__ __forceinline__ int64_t m64_add(int64_t a, int64_t b, int64_t p) {
  int64_t x = a + b;
  return (x >= p) ? x - p : x;
}
__device__ __forceinline__ int64_t m64_mul(int64_t a, int64_t b, int64_t p, uint64_t q) {
  return m64_canon(m64_redc(a, b, p, q), p);
}

// ---------------------------------------------------------------- generic
// Montgomery-domain helpers on canonical uint64 values, dispatching on the
// prime's path.  Used outside the hot loop (setup, combine, finalize).
struct Mont {
  int64_t p;
  uint64_t q;
  int64_t one, r2;
  bool wide;
  __device__ __forceinline__ explicit Mont(const PrimeCtx &c)
      : p((int64_t)c.p), q(c.q), one((int64_t)c.one), r2((int64_t)c.r2), wide(c.flags & 1u) {}
  __device__ __forceinline__ int64_t mul(int64_t a, int64_t b) const {
    if (!wide) return m31_mul((int32_t)a, (int32_t)b, (int32_t)p, (uint32_t)q);
    return m64_mul(a, b, p, q);
  }
  __device__ __forceinline__ int64_t add(int64_t a, int64_t b) const {
    int64_t x = a + b;
    return (x >= p) ? x - p : x;
  }
  __device__ __forceinline__ int64_t sub(int64_t a, int64_t b) const {
    int64_t x = a - b;
    return (x < 0) ? x + p : x;
  }
  __device__ __forceinline__ int64_t to_mont(int64_t a) const { return mul(a, r2); }
  __device__ __forceinline__ int64_t from_mont(int64_t a) const { return mul(a, 1); }
  // plain * plain -> plain
  __device__ __forceinline__ int64_t mulmod(int64_t a, int64_t b) const {
    return mul(mul(a, b), r2);
  }
  __device__ __forceinline__ int64_t pow(int64_t aM, uint64_t e) const {  // Montgomery in/out
    int64_t r = one;
    while (e) {
      if (e & 1) r = mul(r, aM);
      aM = mul(aM, aM);
      e >>= 1;
    }
    return r;
  }
  // (a0 + a1 z)(b0 + b1 z) mod z^2 on Montgomery pairs -- eqn 3.14
  __device__ __forceinline__ void combine(int64_t &a0, int64_t &a1, int64_t b0, int64_t b1) const {
    int64_t n1 = add(mul(a0, b1), mul(a1, b0));
    a0 = mul(a0, b0);
    a1 = n1;
  }
};

}  // namespace wv
