// wv_prime.cuh -- deterministic primality test for n < 2^37, shared by the
// host entry point wv_is_prime and the planner's optional check of the
// caller's prime lists.  64-bit integer operations only, so host and device
// compute the same thing.
#pragma once
#include <cstdint>

namespace wv {

// a b mod m for a, b < m < 2^37: b is split at bit 19 so that every partial
// product stays below 2^57
__host__ __device__ inline uint64_t mulmod37(uint64_t a, uint64_t b, uint64_t m) {
  const uint64_t r = (a * (b >> 19)) % m;                  // < 2^37 * 2^18
  return ((r << 19) + a * (b & ((1ull << 19) - 1))) % m;   // < 2^56 + 2^56
}

__host__ __device__ inline uint64_t powmod37(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod37(r, a, m);
    a = mulmod37(a, a, m);
    e >>= 1;
  }
  return r;
}

// Miller-Rabin with the bases 2, 3, 5, 7, 11, 13, 17: no composite below
// 341,550,071,728,321 (> 2^37) is a strong probable prime to all seven
// (Jaeschke, Math. Comp. 61 (1993)), so for n < 2^37 the test is exact.
__host__ __device__ inline bool is_prime37(uint64_t n) {
  const uint32_t bases[7] = {2, 3, 5, 7, 11, 13, 17};
  if (n < 2) return false;
  for (int i = 0; i < 7; ++i) {
    if (n == bases[i]) return true;
    if (n % bases[i] == 0) return false;
  }
  uint64_t d = n - 1;
  int s = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++s;
  }
  for (int i = 0; i < 7; ++i) {
    uint64_t x = powmod37(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod37(x, x, n);
      if (x == n - 1) {
        witness = false;
        break;
      }
    }
    if (witness) return false;
  }
  return true;
}

}  // namespace wv
