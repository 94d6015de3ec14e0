// wv_search.cu -- step a7: flag the primes of a range whose residue is zero
// (Wolstenholme: p | B_{p-3}; Vandiver: p | E_{p-3}; Sec. 3 and Sec. 5) and,
// optionally, the near misses |<r>_p| < near of Tables 1-2, where <r>_p is the
// representative of r mod p in (-p/2, p/2].
//
// The range is processed in windows: sieve the window on the device, compute
// both residues for its primes, flag, and compact the flagged primes in
// ascending order (exclusive scan of the flags, then scatter).  The histogram
// mode (Sec. 3 "Results", the 2000-bin histogram of <B_{p-3}>_p / p) replaces
// the flag/compact epilogue by a binning kernel over the same windows.
#include "wv_internal.h"

namespace wv {

constexpr uint64_t kSearchWindow = 1ull << 25;  // integers per window

__device__ __forceinline__ bool near_zero(uint64_t r, uint64_t p, uint64_t near) {
  if (r == WV_RESIDUE_INVALID) return false;
  // |<r>_p| < near  <=>  r < near  or  p - r < near
  return r < near || (p - r) < near;
}

__global__ void k_flag(const uint64_t *primes, const uint64_t *rb, const uint64_t *re, size_t n,
                       uint64_t near, uint32_t *kind, uint32_t *flag) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t p = primes[i];
  uint32_t k = 0;
  if (p >= 5) {
    if (rb[i] == 0) k |= WV_KIND_BERNOULLI;
    if (re[i] == 0) k |= WV_KIND_EULER;
    if (near) {
      if (near_zero(rb[i], p, near)) k |= WV_KIND_NEAR_B;
      if (near_zero(re[i], p, near)) k |= WV_KIND_NEAR_E;
    }
  }
  kind[i] = k;
  flag[i] = k ? 1u : 0u;
}

__global__ void k_scatter_hits(const uint64_t *primes, const uint32_t *kind, const uint32_t *off,
                               size_t n, uint64_t base, wv_hit *hits, uint64_t cap) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || kind[i] == 0) return;
  uint64_t slot = base + off[i];
  if (slot < cap) {
    wv_hit h;
    h.p = primes[i];
    h.kind = kind[i];
    h.pad = 0;
    hits[slot] = h;
  }
}

__global__ void k_copy_u64(const uint64_t *src, uint64_t *dst, size_t n, uint64_t base, uint64_t cap) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && base + i < cap) dst[base + i] = src[i];
}

// Bin of <r>_p / p: with u = <r>_p / p + 1/2 = (2<r>_p + p) / (2p) in (0, 1),
// bin = floor(u bins), i.e. bins [b / bins, (b + 1) / bins) of u.  Per-block
// counts in shared memory (bins <= kHistShared), then one atomic per bin.
constexpr uint32_t kHistShared = 8192;

__global__ void k_hist(const uint64_t *primes, const uint64_t *res, size_t n, uint32_t bins,
                       unsigned long long *hist) {
  extern __shared__ uint32_t sh[];
  const bool local = bins <= kHistShared;
  if (local)
    for (uint32_t b = threadIdx.x; b < bins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t p = primes[i], r = res[i];
    if (p < 5 || r >= p) continue;  // invalid slots carry WV_RESIDUE_INVALID
    const uint64_t num = (r > p / 2) ? 2 * r - p : 2 * r + p;  // 2 <r>_p + p, in [1, 2p)
    const uint32_t b = (uint32_t)(num * bins / (2 * p));
    if (local) atomicAdd(&sh[b], 1u);
    else atomicAdd(&hist[b], 1ull);
  }
  if (!local) return;
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < bins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

struct HistOut {
  uint32_t bins = 0;
  unsigned long long *b = nullptr, *e = nullptr;
};

static wv_status search_impl(uint64_t lo, uint64_t hi, uint64_t near, wv_hit *d_hits, size_t cap,
                             size_t *n_hits, uint64_t *d_primes_out, uint64_t *d_rb_out,
                             uint64_t *d_re_out, size_t cap_primes, size_t *n_primes,
                             const wv_options *opt, cudaStream_t s, const HistOut *hist = nullptr) {
  if (!n_hits) return set_error(WV_EINVAL, "n_hits is NULL");
  if (cap && !d_hits) return set_error(WV_EINVAL, "d_hits is NULL with cap > 0");
  if (hi > WV_P_MAX || lo > hi) return set_error(WV_EINVAL, "range [%llu, %llu) invalid",
                                                 (unsigned long long)lo, (unsigned long long)hi);
  ResidueConfig cfg;
  WV_CHECK(resolve_config(opt, true, true, &cfg));
  {  // congruences the caller left open: the cheapest for primes below hi
    int cb = cfg.cong_b, ce = cfg.cong_e;
    cong_for_range(hi, &cb, &ce);
    if (cfg.cong_auto_b) cfg.cong_b = cb;
    if (cfg.cong_auto_e) cfg.cong_e = ce;
  }
  if (lo < 5) lo = 5;
  uint64_t hits_total = 0, primes_total = 0;
  if (hi > lo) {
    const uint64_t win = (hi - lo < kSearchWindow) ? hi - lo : kSearchWindow;
    const size_t maxp = (size_t)(win / 2 + 2);  // odd numbers in a window bound its primes
    Scratch sc(s);
    uint64_t *pr = nullptr, *rb = nullptr, *re = nullptr;
    uint32_t *kind = nullptr, *flag = nullptr, *off = nullptr, *tmp = nullptr, *tot = nullptr;
    WV_CHECK(sc.get(&pr, maxp));
    WV_CHECK(sc.get(&rb, maxp));
    WV_CHECK(sc.get(&re, maxp));
    WV_CHECK(sc.get(&kind, maxp));
    WV_CHECK(sc.get(&flag, maxp));
    WV_CHECK(sc.get(&off, maxp));
    WV_CHECK(sc.get(&tmp, scan_tmp_elems(maxp)));
    WV_CHECK(sc.get(&tot, 1));
    for (uint64_t w_lo = lo; w_lo < hi; w_lo += win) {
      const uint64_t w_hi = (hi - w_lo < win) ? hi : w_lo + win;
      uint64_t np = 0;
      WV_CHECK(sieve_device(w_lo, w_hi, pr, maxp, &np, s));
      if (np == 0) continue;
      WV_CHECK(residues_device(pr, np, rb, re, cfg, s));
      const unsigned g = (unsigned)((np + 255) / 256);
      if (hist) {
        const unsigned hg = g < 1024 ? g : 1024;
        const size_t shb = hist->bins <= kHistShared ? hist->bins * sizeof(uint32_t) : 0;
        if (hist->b) WV_LAUNCH("hist", k_hist, hg, 256, shb, s, pr, rb, (size_t)np, hist->bins, hist->b);
        if (hist->e) WV_LAUNCH("hist", k_hist, hg, 256, shb, s, pr, re, (size_t)np, hist->bins, hist->e);
        primes_total += np;
        continue;
      }
      WV_LAUNCH("search_flag", k_flag, g, 256, 0, s, pr, rb, re, (size_t)np, near, kind, flag);
      WV_CHECK(scan_exclusive_u32(flag, off, np, tot, tmp, s));
      WV_LAUNCH("search_scatter", k_scatter_hits, g, 256, 0, s, pr, kind, off, (size_t)np,
                hits_total, d_hits, (uint64_t)cap);
      if (cap_primes) {
        if (d_primes_out)
          WV_LAUNCH("search_copy", k_copy_u64, g, 256, 0, s, pr, d_primes_out, (size_t)np,
                    primes_total, (uint64_t)cap_primes);
        if (d_rb_out)
          WV_LAUNCH("search_copy", k_copy_u64, g, 256, 0, s, rb, d_rb_out, (size_t)np,
                    primes_total, (uint64_t)cap_primes);
        if (d_re_out)
          WV_LAUNCH("search_copy", k_copy_u64, g, 256, 0, s, re, d_re_out, (size_t)np,
                    primes_total, (uint64_t)cap_primes);
      }
      uint32_t h = 0;
      WV_CUDA(cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s));
      WV_CUDA(cudaStreamSynchronize(s));
      hits_total += h;
      primes_total += np;
    }
  }
  *n_hits = (size_t)hits_total;
  if (n_primes) *n_primes = (size_t)primes_total;
  if (hits_total > cap)
    return set_error(WV_ERANGE, "%llu hits, capacity %zu", (unsigned long long)hits_total, cap);
  if (cap_primes && primes_total > cap_primes)
    return set_error(WV_ERANGE, "%llu primes, capacity %zu", (unsigned long long)primes_total,
                     cap_primes);
  return WV_OK;
}

}  // namespace wv

using namespace wv;

extern "C" {

wv_status wv_search(uint64_t lo, uint64_t hi, wv_hit *d_hits, size_t cap, size_t *n_hits,
                    wv_stream stream) {
  clear_error();
  return search_impl(lo, hi, 0, d_hits, cap, n_hits, nullptr, nullptr, nullptr, 0, nullptr,
                     nullptr, (cudaStream_t)stream);
}

wv_status wv_histogram(uint64_t lo, uint64_t hi, uint32_t bins, unsigned long long *d_hist_b,
                       unsigned long long *d_hist_e, size_t *n_primes, wv_stream stream) {
  clear_error();
  if (bins < 1 || bins > (1u << 20)) return set_error(WV_EINVAL, "bins=%u not in [1, 2^20]", bins);
  if (!d_hist_b && !d_hist_e) return set_error(WV_EINVAL, "no histogram output");
  HistOut h;
  h.bins = bins;
  h.b = d_hist_b;
  h.e = d_hist_e;
  size_t nh = 0, np = 0;
  WV_CHECK(search_impl(lo, hi, 0, nullptr, 0, &nh, nullptr, nullptr, nullptr, 0, &np, nullptr,
                       (cudaStream_t)stream, &h));
  WV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (n_primes) *n_primes = np;
  return WV_OK;
}

wv_status wv_search_ex(uint64_t lo, uint64_t hi, uint64_t near, wv_hit *d_hits, size_t cap,
                       size_t *n_hits, uint64_t *d_primes, uint64_t *d_res_b, uint64_t *d_res_e,
                       size_t cap_primes, size_t *n_primes, const wv_options *opt,
                       wv_stream stream) {
  clear_error();
  if (cap_primes && !d_primes && !d_res_b && !d_res_e)
    return set_error(WV_EINVAL, "cap_primes > 0 but no prime/residue output");
  return search_impl(lo, hi, near, d_hits, cap, n_hits, d_primes, d_res_b, d_res_e, cap_primes,
                     n_primes, opt, (cudaStream_t)stream);
}

}  // extern "C"
