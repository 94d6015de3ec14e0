// wv_diag.cu -- integer-pipe throughput probes (see include/wv_diag.h).
//
// Each thread runs 8 independent chains of one instruction kind; every block
// records its elapsed SM cycles (clock64).  With one full wave of resident
// blocks, per-SM throughput = (blocks per SM x threads x iters x 8) / cycles.
#include "../../include/wv_diag.h"
#include "wv_internal.h"

namespace wv {

constexpr int kDiagThreads = 256;

template <int OP>
__global__ void __launch_bounds__(kDiagThreads) k_diag(int iters, uint32_t seed, uint64_t *cycles,
                                                       uint32_t *sink) {
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1) + i * 0x9e3779b9u;
  const uint32_t x = seed | 1u, y = seed ^ 0x5bd1e995u;
  __syncthreads();
  const uint64_t t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (OP == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(x), "r"(y));
      if (OP == 1) asm volatile("mul.hi.s32 %0, %0, %1;" : "+r"(a[i]) : "r"(x));
      if (OP == 2) {
        uint64_t w;
        asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(w) : "r"(a[i]), "r"(x));
        a[i] = (uint32_t)(w >> 32) ^ (uint32_t)w;
      }
      if (OP == 3) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(x));
      if (OP == 4) asm volatile("min.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(y));
      if (OP == 9) {
        int64_t w;
        asm volatile("mul.wide.s32 %0, %1, %2;" : "=l"(w) : "r"(a[i]), "r"(x));
        a[i] = (uint32_t)(w >> 32) ^ (uint32_t)w;
      }
      if (OP == 10) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(x));
      if (OP == 11) {  // one signed Montgomery product: wide, lo * q, hi(m p), subtract
        int64_t w;
        uint32_t m, u;
        asm volatile("mul.wide.s32 %0, %1, %2;" : "=l"(w) : "r"(a[i]), "r"(x));
        asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(m) : "r"((uint32_t)w), "r"(y));
        asm volatile("mul.hi.s32 %0, %1, %2;" : "=r"(u) : "r"(m), "r"(x));
        a[i] = (uint32_t)(w >> 32) - u;
      }
      if (OP == 12) {  // Shoup product: hi(c t'), c t - q p
        uint32_t qq, r;
        asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(qq) : "r"(a[i]), "r"(y));
        asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(a[i]), "r"(x));
        asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(r) : "r"(qq), "r"(0u - x));
        a[i] = r;
      }
    }
  }
  __syncthreads();
  const uint64_t t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) acc ^= a[i];
  if (acc == 0x12345678u) sink[0] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The hot-loop term body of the p < 2^30 accumulation (2 independent chains).
template <bool CUBES, int AR>
__global__ void __launch_bounds__(kDiagThreads) k_diag_term(int iters, uint32_t seed, uint64_t *cycles,
                                                            uint32_t *sink) {
  const int32_t p = 1062232319;  // < 2^30
  uint32_t q = (uint32_t)p;
  for (int i = 0; i < 4; ++i) q *= 2u - (uint32_t)p * q;
  const uint32_t up = (uint32_t)p;
  int32_t c0[2], c1[2], t[2], d1[2], d2[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    c0[k] = (int32_t)((seed + threadIdx.x * 7u + k) % up);
    c1[k] = 0;
    t[k] = (int32_t)((seed * 3u + threadIdx.x + k) % up);
    d1[k] = (int32_t)((seed * 5u + threadIdx.x) % up);
    d2[k] = (int32_t)((seed * 11u + k) % up);
  }
  __syncthreads();
  const uint64_t t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (AR == 1) {
        const uint32_t tq = (uint32_t)t[k] * q;
        const int32_t m0 = (int32_t)((uint32_t)c0[k] * tq);
        const int32_t m1 = (int32_t)((uint32_t)c1[k] * tq);
        const int32_t h0 = __mulhi(c0[k], t[k]);
        const int32_t h1 = __mulhi(c1[k], t[k]);
        const int32_t n1 = h1 - __mulhi(m1, p) + c0[k];
        c0[k] = h0 - __mulhi(m0, p);
        c1[k] = n1;
      } else {
        const int64_t w0 = (int64_t)c0[k] * (int64_t)t[k];
        const int64_t w1 = (int64_t)c1[k] * (int64_t)t[k];
        const int32_t m0 = (int32_t)((uint32_t)w0 * q);
        const int32_t m1 = (int32_t)((uint32_t)w1 * q);
        const int32_t n1 = (int32_t)(w1 >> 32) - __mulhi(m1, p) + c0[k];
        c0[k] = (int32_t)(w0 >> 32) - __mulhi(m0, p);
        c1[k] = n1;
      }
      uint32_t x = (uint32_t)t[k] + (uint32_t)d1[k];
      t[k] = (int32_t)min(x, x - up);
      if (CUBES) {
        x = (uint32_t)d1[k] + (uint32_t)d2[k];
        d1[k] = (int32_t)min(x, x - up);
        x = (uint32_t)d2[k] + 6u;
        d2[k] = (int32_t)min(x, x - up);
      } else {
        d1[k] += 2;
      }
    }
  }
  __syncthreads();
  const uint64_t t1 = clock64();
  uint32_t acc = (uint32_t)(c0[0] ^ c1[0] ^ c0[1] ^ c1[1] ^ t[0] ^ t[1]);
  if (acc == 0x12345678u) sink[0] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Euler hot-loop body with Shoup products: c t mod p = c t - hi(c t') p with
// t' = floor(t 2^32 / p) carried along the forward differences.
__global__ void __launch_bounds__(kDiagThreads) k_diag_shoup_e(int iters, uint32_t seed,
                                                               uint64_t *cycles, uint32_t *sink) {
  const uint32_t p = 1062232319u, np = 0u - p;
  uint32_t c0[2], c1[2], t[2], tp[2], th[2], d[2], dp[2], dh[2];
  const uint32_t twop = (uint32_t)((2ull << 32) / p) + 1u, twoh = (uint32_t)((2ull << 32) % p);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    c0[k] = (seed + threadIdx.x * 7u + k) % p; c1[k] = 0;
    t[k] = (seed * 3u + threadIdx.x + k) % p; tp[k] = t[k] * 3u; th[k] = t[k] >> 1;
    d[k] = (seed * 5u + threadIdx.x) % p; dp[k] = d[k] * 5u; dh[k] = d[k] >> 2;
  }
  __syncthreads();
  const uint64_t t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t q0 = __umulhi(c0[k], tp[k]);
      const uint32_t q1 = __umulhi(c1[k], tp[k]);
      const uint32_t n1 = c1[k] * t[k] + c0[k] + q1 * np;
      c0[k] = c0[k] * t[k] + q0 * np;
      c1[k] = n1;
      // t, t', t^ += d, d', d^
      int32_t sg = (int32_t)(th[k] + dh[k] - p);
      int32_t sgn = sg >> 31;
      th[k] = (uint32_t)sg + (p & (uint32_t)sgn);
      tp[k] = tp[k] + dp[k] + (uint32_t)sgn;
      uint32_t x = t[k] + d[k];
      t[k] = min(x, x - p);
      // d, d', d^ += 2, 2', 2^
      d[k] += 2u;
      sg = (int32_t)(dh[k] + twoh - p);
      sgn = sg >> 31;
      dh[k] = (uint32_t)sg + (p & (uint32_t)sgn);
      dp[k] = dp[k] + twop + (uint32_t)sgn;
    }
  }
  __syncthreads();
  const uint64_t t1 = clock64();
  uint32_t acc = c0[0] ^ c1[0] ^ c0[1] ^ c1[1] ^ t[0] ^ tp[1] ^ dp[0] ^ th[1];
  if (acc == 0x12345678u) sink[0] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace wv

using namespace wv;

extern "C" wv_status wv_diag_throughput(int op, int iters, double *per_clk) {
  clear_error();
  if (!per_clk || iters < 1 || op < 0 || op > 13) return set_error(WV_EINVAL, "bad diag arguments");
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));
  void (*kern)(int, uint32_t, uint64_t *, uint32_t *) = nullptr;
  switch (op) {
    case 0: kern = k_diag<0>; break;
    case 1: kern = k_diag<1>; break;
    case 2: kern = k_diag<2>; break;
    case 3: kern = k_diag<3>; break;
    case 4: kern = k_diag<4>; break;
    case 5: kern = k_diag_term<true, 1>; break;
    case 6: kern = k_diag_term<false, 1>; break;
    case 7: kern = k_diag_term<true, 2>; break;
    case 8: kern = k_diag_term<false, 2>; break;
    case 9: kern = k_diag<9>; break;
    case 10: kern = k_diag<10>; break;
    case 11: kern = k_diag<11>; break;
    case 12: kern = k_diag<12>; break;
    default: kern = k_diag_shoup_e; break;
  }
  int occ = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kDiagThreads, 0));
  if (occ < 1) occ = 1;
  const int blocks = dev->sms * occ;
  uint64_t *cyc = nullptr;
  uint32_t *sink = nullptr;
  WV_CUDA(cudaMalloc(&cyc, blocks * sizeof(uint64_t)));
  WV_CUDA(cudaMalloc(&sink, sizeof(uint32_t)));
  kern<<<blocks, kDiagThreads>>>(iters, 12345u, cyc, sink);  // warm-up
  kern<<<blocks, kDiagThreads>>>(iters, 777u, cyc, sink);
  cudaError_t e = cudaDeviceSynchronize();
  uint64_t *h = new uint64_t[blocks];
  if (e == cudaSuccess) e = cudaMemcpy(h, cyc, blocks * sizeof(uint64_t), cudaMemcpyDeviceToHost);
  cudaFree(cyc);
  cudaFree(sink);
  if (e != cudaSuccess) {
    delete[] h;
    return cuda_fail(e, "wv_diag_throughput");
  }
  uint64_t mx = 0;
  for (int i = 0; i < blocks; ++i) mx = h[i] > mx ? h[i] : mx;
  delete[] h;
  const bool term = (op >= 5 && op <= 8) || op == 13;
  const double per_thread = term ? 2.0 * iters : 8.0 * iters;  // ops (or terms) per thread
  *per_clk = (double)occ * kDiagThreads * per_thread / (double)mx;
  return WV_OK;
}
