// wv_sieve.cu -- segmented sieve of Eratosthenes on the GPU (step a1).
//
// The paper enumerates the primes of each search interval on the CPU (with
// primesieve, Sec. 3 "Results" and Sec. 5); here the enumeration runs on the
// device so the prime list never leaves HBM.
//
// Layout: a window [lo, hi) is represented by the odd numbers n = 2v + 1 with
// odd index v in [lo/2, hi/2).  One CTA sieves one segment of kSegBits odd
// indices in a shared-memory bitset (bit set = composite), crossing off the
// odd multiples q*m (m odd, m >= q) of every odd base prime q with q^2 < hi.
// Pass 1 writes the per-segment prime count (and, when the primes are to be
// listed, the segment's bit words to global memory); an exclusive scan of the
// counts gives each segment's output offset; pass 2 expands the stored words
// into ascending prime values.  The prime 2 is prepended on the host side of
// the launch sequence when lo <= 2 < hi.
#include "wv_internal.h"

namespace wv {

constexpr int kSegBits = 1 << 18;           // odd indices per segment (2^19 integers)
constexpr int kSegWords = kSegBits / 32;   // 8192 words = 32 KB shared memory
constexpr int kSieveThreads = 512;
constexpr int kWarpPrimeLimit = 1024;       // base primes q < this are marked warp-cooperatively

// ---------------------------------------------------------------- base primes
// One CTA: odd primes 3 <= q < limit by a plain sieve in shared memory.
__global__ void k_base_primes(uint32_t *out, uint32_t *count, uint32_t limit) {
  extern __shared__ uint32_t bits[];  // bit v <-> odd number 2v+1, set = composite
  const uint32_t nodd = limit / 2;    // odd numbers 1, 3, ..., < limit
  const uint32_t words = (nodd + 31) / 32;
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0;
  __syncthreads();
  if (threadIdx.x == 0) bits[0] |= 1u;  // 1 is not prime
  __syncthreads();
  for (uint32_t q = 3; q * q < limit; q += 2) {
    uint32_t v = q / 2;
    bool prime = !((bits[v >> 5] >> (v & 31)) & 1u);
    __syncthreads();
    if (prime) {
      // odd multiples q*m, m = q, q+2, ...  -> indices (q*m-1)/2, step q
      for (uint32_t idx = (q * q) / 2 + threadIdx.x * q; idx < nodd; idx += blockDim.x * q)
        atomicOr(&bits[idx >> 5], 1u << (idx & 31));
    }
    __syncthreads();
  }
  // ordered compaction, one word per thread per round
  __shared__ uint32_t sw[33];
  __shared__ uint32_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (uint32_t w0 = 0; w0 < words; w0 += blockDim.x) {
    uint32_t w = w0 + threadIdx.x;
    uint32_t live = 0;
    if (w < words) {
      live = ~bits[w];
      uint32_t hi_idx = (w + 1) * 32;
      if (hi_idx > nodd) live &= (nodd - w * 32 >= 32) ? 0xffffffffu : ((1u << (nodd - w * 32)) - 1u);
    }
    uint32_t c = __popc(live);
    // block exclusive scan of c
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t v = (lane < (int)(blockDim.x >> 5)) ? sw[lane] : 0u;
      uint32_t vx = v;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, vx, o);
        if (lane >= o) vx += y;
      }
      sw[lane] = vx - v;
      if (lane == 31) sw[32] = vx;
    }
    __syncthreads();
    uint32_t off = base + sw[warp] + x - c;
    while (live) {
      int b = __ffs(live) - 1;
      live &= live - 1;
      out[off++] = 2u * (w * 32 + b) + 1u;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += sw[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

wv_status launch_base_primes(uint32_t *out, uint32_t *count, uint32_t limit) {
  size_t smem = ((limit / 2 + 31) / 32) * sizeof(uint32_t);
  WV_CUDA(cudaFuncSetAttribute(k_base_primes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  WV_LAUNCH("sieve_base_primes", k_base_primes, 1, 1024, smem, (cudaStream_t)0, out, count, limit);
  WV_CUDA(cudaDeviceSynchronize());
  return WV_OK;
}

// ---------------------------------------------------------------- segments
struct SieveArgs {
  uint64_t v_lo, v_hi;          // odd-index window [v_lo, v_hi)
  const uint32_t *base;         // odd base primes, ascending
  uint32_t n_base;              // only those with q^2 < hi are used
  uint32_t *seg_count;          // per segment prime count
  uint32_t *seg_words;          // optional: kSegWords words per segment (1 = prime)
};

__global__ void __launch_bounds__(kSieveThreads) k_sieve_segment(SieveArgs a) {
  __shared__ uint32_t bits[kSegWords];  // set = composite
  const uint64_t s_lo = a.v_lo + (uint64_t)blockIdx.x * kSegBits;
  uint64_t s_hi = s_lo + kSegBits;
  if (s_hi > a.v_hi) s_hi = a.v_hi;
  const uint32_t nbits = (uint32_t)(s_hi - s_lo);
  for (int w = threadIdx.x; w < kSegWords; w += blockDim.x) bits[w] = 0;
  __syncthreads();
  if (threadIdx.x == 0 && s_lo == 0) atomicOr(&bits[0], 1u);  // odd index 0 is the number 1
  const uint64_t n_hi = 2 * s_hi + 1;                  // numbers below this are in play
  const uint64_t n_lo = 2 * s_lo + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  // small base primes: one warp per prime, lanes stride over the multiples
  for (uint32_t i = warp; i < a.n_base; i += nwarps) {
    uint64_t q = a.base[i];
    if (q >= kWarpPrimeLimit) break;
    if (q * q >= n_hi) break;
    uint64_t m = (n_lo + q - 1) / q;  // first multiple >= n_lo
    if (m < q) m = q;
    if ((m & 1) == 0) ++m;
    uint64_t idx = (q * m - 1) / 2 - s_lo;  // odd index relative to the segment
    for (uint64_t k = idx + (uint64_t)lane * q; k < nbits; k += 32 * q)
      atomicOr(&bits[k >> 5], 1u << (k & 31));
  }
  // larger base primes: one thread per prime
  for (uint32_t i = threadIdx.x; i < a.n_base; i += blockDim.x) {
    uint64_t q = a.base[i];
    if (q < kWarpPrimeLimit) continue;
    if (q * q >= n_hi) break;
    uint64_t m = (n_lo + q - 1) / q;
    if (m < q) m = q;
    if ((m & 1) == 0) ++m;
    uint64_t idx = (q * m - 1) / 2 - s_lo;
    for (uint64_t k = idx; k < nbits; k += q) atomicOr(&bits[k >> 5], 1u << (k & 31));
  }
  __syncthreads();

  uint32_t cnt = 0;
  for (uint32_t w = threadIdx.x; w < kSegWords; w += blockDim.x) {
    uint32_t live = ~bits[w];
    uint32_t b0 = w * 32;
    if (b0 >= nbits) live = 0;
    else if (nbits - b0 < 32) live &= (1u << (nbits - b0)) - 1u;
    cnt += __popc(live);
    if (a.seg_words) a.seg_words[(uint64_t)blockIdx.x * kSegWords + w] = live;
  }
  // block reduce
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __shared__ uint32_t red[32];
  if (lane == 0) red[warp] = cnt;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = (lane < nwarps) ? red[lane] : 0u;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) a.seg_count[blockIdx.x] = v;
  }
}

// Expand stored words into prime values at the scanned segment offsets.
__global__ void __launch_bounds__(kSieveThreads)
    k_sieve_expand(uint64_t v_lo, const uint32_t *seg_words, const uint64_t *seg_off,
                   uint64_t shift, uint64_t *out, uint64_t cap) {
  __shared__ uint32_t sw[33];
  __shared__ uint64_t base;
  if (threadIdx.x == 0) base = seg_off[blockIdx.x] + shift;
  __syncthreads();
  const uint64_t s_lo = v_lo + (uint64_t)blockIdx.x * kSegBits;
  const uint32_t *words = seg_words + (uint64_t)blockIdx.x * kSegWords;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w0 = 0; w0 < kSegWords; w0 += blockDim.x) {
    int w = w0 + threadIdx.x;
    uint32_t live = (w < kSegWords) ? words[w] : 0u;
    uint32_t c = __popc(live);
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t v = (lane < (int)(blockDim.x >> 5)) ? sw[lane] : 0u;
      uint32_t vx = v;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, vx, o);
        if (lane >= o) vx += y;
      }
      sw[lane] = vx - v;
      if (lane == 31) sw[32] = vx;
    }
    __syncthreads();
    uint64_t off = base + sw[warp] + x - c;
    while (live) {
      int b = __ffs(live) - 1;
      live &= live - 1;
      if (off < cap) out[off] = 2 * (s_lo + (uint64_t)w * 32 + b) + 1;
      ++off;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += sw[32];
    __syncthreads();
  }
}

__global__ void k_put_two(uint64_t *out, uint64_t cap) {
  if (cap > 0) out[0] = 2;
}

__global__ void k_widen(const uint32_t *in, uint64_t *out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}
wv_status widen_u32(const uint32_t *in, uint64_t *out, size_t n, cudaStream_t s) {
  if (!n) return WV_OK;
  WV_LAUNCH("widen", k_widen, (unsigned)((n + 255) / 256), 256, 0, s, in, out, n);
  return WV_OK;
}

// Pass 1 (+ optional pass 2) for the window; count (host) = number of primes.
wv_status sieve_device(uint64_t lo, uint64_t hi, uint64_t *d_out, size_t cap,
                       uint64_t *count_host, cudaStream_t s) {
  if (hi > WV_P_MAX || lo > hi)
    return set_error(WV_EINVAL, "sieve range [%llu, %llu) invalid (hi <= 2^37 required)",
                     (unsigned long long)lo, (unsigned long long)hi);
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));
  const bool two = (lo <= 2 && 2 < hi);
  const uint64_t v_lo = lo / 2, v_hi = hi / 2;
  uint64_t total = two ? 1 : 0;
  if (v_hi > v_lo) {
    const uint64_t nseg = (v_hi - v_lo + kSegBits - 1) / kSegBits;
    if (nseg > (1ull << 31)) return set_error(WV_EINVAL, "sieve window too large");
    const bool list = (d_out != nullptr && cap > 0);
    // in list mode the bit words are stored; keep each batch of segments to ~1 GB
    const uint64_t batch = list ? (uint64_t)(1ull << 30) / (kSegWords * 4) : nseg;
    Scratch sc(s);
    uint32_t *cnt32 = nullptr, *words = nullptr;
    uint64_t *cnt64 = nullptr, *off = nullptr, *tmp = nullptr, *dtot = nullptr;
    const uint64_t bseg = batch < nseg ? batch : nseg;
    WV_CHECK(sc.get(&cnt32, bseg));
    WV_CHECK(sc.get(&cnt64, bseg));
    WV_CHECK(sc.get(&off, bseg));
    WV_CHECK(sc.get(&tmp, scan_tmp_elems(bseg)));
    WV_CHECK(sc.get(&dtot, 1));
    if (list) WV_CHECK(sc.get(&words, bseg * kSegWords));
    uint64_t h_tot = 0;
    wv_status st = WV_OK;
    for (uint64_t b0 = 0; b0 < nseg && st == WV_OK; b0 += bseg) {
      uint64_t nb = (nseg - b0 < bseg) ? nseg - b0 : bseg;
      SieveArgs a;
      a.v_lo = v_lo + b0 * kSegBits;
      a.v_hi = v_hi;
      a.base = dev->base_primes;
      a.n_base = dev->n_base;
      a.seg_count = cnt32;
      a.seg_words = list ? words : nullptr;
      prof_begin("sieve_segment", s);
      k_sieve_segment<<<(unsigned)nb, kSieveThreads, 0, s>>>(a);
      prof_end("sieve_segment", s);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { st = cuda_fail(e, "sieve_segment"); break; }
      // widen counts to 64 bit and scan
      e = cudaMemsetAsync(cnt64, 0, nb * sizeof(uint64_t), s);
      if (e != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
      st = widen_u32(cnt32, cnt64, nb, s);
      if (st != WV_OK) break;
      st = scan_exclusive_u64(cnt64, off, nb, dtot, tmp, s);
      if (st != WV_OK) break;
      if (list) {
        prof_begin("sieve_expand", s);
        k_sieve_expand<<<(unsigned)nb, kSieveThreads, 0, s>>>(a.v_lo, words, off, total, d_out, cap);
        prof_end("sieve_expand", s);
        e = cudaGetLastError();
        if (e != cudaSuccess) { st = cuda_fail(e, "sieve_expand"); break; }
      }
      e = cudaMemcpyAsync(&h_tot, dtot, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { st = cuda_fail(e, "sieve count"); break; }
      total += h_tot;
    }
    if (st != WV_OK) return st;
  }
  if (two && d_out && cap > 0) WV_LAUNCH("sieve_put_two", k_put_two, 1, 1, 0, s, d_out, cap);
  if (count_host) *count_host = total;
  return WV_OK;
}

}  // namespace wv

using namespace wv;

extern "C" wv_status wv_sieve(uint64_t lo, uint64_t hi, uint64_t *d_out, size_t cap,
                              size_t *n_out, wv_stream stream) {
  clear_error();
  if (!n_out) return set_error(WV_EINVAL, "n_out is NULL");
  if (cap > 0 && !d_out) return set_error(WV_EINVAL, "d_out is NULL with cap > 0");
  uint64_t count = 0;
  WV_CHECK(sieve_device(lo, hi, cap ? d_out : nullptr, cap, &count, (cudaStream_t)stream));
  // in list mode the prime 2 shifts every odd prime by one slot: handled by `shift`
  *n_out = (size_t)count;
  if (count > cap) return set_error(WV_ERANGE, "%llu primes in range, capacity %zu",
                                    (unsigned long long)count, cap);
  return WV_OK;
}

extern "C" wv_status wv_sieve_count(uint64_t lo, uint64_t hi, uint64_t *count, wv_stream stream) {
  clear_error();
  if (!count) return set_error(WV_EINVAL, "count is NULL");
  return sieve_device(lo, hi, nullptr, 0, count, (cudaStream_t)stream);
}
