// wv_runtime.cu -- errors, per-device state, scratch pool, launch profiling,
// device-wide scans, and the host-side congruence-table API.
#include "wv_prime.cuh"
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "wv_internal.h"
#include "wv_tables.h"

namespace wv {

// ================================================================ errors
static thread_local std::string g_err;

wv_status set_error(wv_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}
void clear_error() { g_err.clear(); }
wv_status cuda_fail(cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(WV_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return set_error(WV_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ================================================================ devices
static std::mutex g_dev_mu;
static DeviceState g_dev[64];

wv_status launch_base_primes(uint32_t *out, uint32_t *count, uint32_t limit);

wv_status device_state(DeviceState **out) {
  int dev = 0;
  WV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(WV_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceState &d = g_dev[dev];
  if (d.device != dev) {
    cudaDeviceProp prop;
    WV_CUDA(cudaGetDeviceProperties(&prop, dev));
    d.sms = prop.multiProcessorCount;
    d.cc_major = prop.major;
    d.cc_minor = prop.minor;
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    WV_CUDA(cudaMemPoolCreate(&d.pool, &pp));
    uint64_t thresh = UINT64_MAX;  // keep freed blocks cached in the pool
    WV_CUDA(cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thresh));
    // base primes: odd primes up to sqrt(2^37) ~ 370727.6, computed once
    const uint32_t limit = 370728;
    uint32_t *buf = nullptr, *cnt = nullptr;
    WV_CUDA(cudaMalloc(&buf, 40000 * sizeof(uint32_t)));
    WV_CUDA(cudaMalloc(&cnt, sizeof(uint32_t)));
    WV_CUDA(cudaMemset(cnt, 0, sizeof(uint32_t)));
    WV_CHECK(launch_base_primes(buf, cnt, limit));
    uint32_t n = 0;
    WV_CUDA(cudaMemcpy(&n, cnt, sizeof n, cudaMemcpyDeviceToHost));
    WV_CUDA(cudaFree(cnt));
    d.base_primes = buf;
    d.n_base = n;
    WV_CHECK(cong_upload(&d));
    d.device = dev;
  }
  *out = &d;
  return WV_OK;
}

// ================================================================ scratch
wv_status scratch_alloc(void **ptr, size_t bytes, cudaStream_t s) {
  DeviceState *d = nullptr;
  WV_CHECK(device_state(&d));
  cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes ? bytes : 256, d->pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return set_error(WV_ENOMEM, "scratch allocation of %zu bytes failed: %s", bytes,
                     cudaGetErrorString(e));
  }
  return WV_OK;
}
void scratch_free(void *ptr, cudaStream_t s) {
  if (ptr) cudaFreeAsync(ptr, s);
}

// ================================================================ profiling
namespace {
struct ProfEntry {
  uint64_t launches = 0;
  double total_ms = 0;
};
struct PendingEvent {
  std::string name;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<std::string> g_prof_names;
std::map<std::string, ProfEntry> g_prof;
std::vector<PendingEvent> g_pending;
std::vector<cudaEvent_t> g_event_pool;
uint64_t g_launches = 0;
thread_local cudaEvent_t t_begin_ev = nullptr;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void prof_begin(const char *name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ++g_launches;
  auto it = g_prof.find(name);
  if (it == g_prof.end()) {
    g_prof_names.push_back(name);
    it = g_prof.emplace(name, ProfEntry{}).first;
  }
  it->second.launches++;
  if (g_prof_on) {
    // no timing events inside a stream capture: they would become graph nodes
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      t_begin_ev = take_event();
      cudaEventRecord(t_begin_ev, s);
    }
  }
}
void prof_end(const char *name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_on && t_begin_ev) {
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    g_pending.push_back({name, t_begin_ev, e});
    t_begin_ev = nullptr;
  }
}

// ================================================================ scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *smem_warp, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : T(0);
    T wx = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, wx, o);
      if (lane >= o) wx += y;
    }
    smem_warp[lane] = wx - w;  // exclusive warp offsets
    if (lane == 31) smem_warp[32] = wx;
  }
  __syncthreads();
  T res = smem_warp[warp] + x - v;
  *total = smem_warp[32];
  __syncthreads();
  return res;
}

template <typename T>
__global__ void k_scan_tiles(const T *in, T *out, size_t n, T *tile_sums) {
  __shared__ T sw[33];
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : T(0);
    sum += v[i];
  }
  T tot;
  T off = block_exclusive_scan<T>(sum, sw, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = off;
    off += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in place, total to *d_total
template <typename T>
__global__ void k_scan_top(T *sums, size_t m, T *d_total) {
  __shared__ T sw[33];
  T carry = 0;
  for (size_t b = 0; b < m; b += blockDim.x) {
    size_t i = b + threadIdx.x;
    T v = (i < m) ? sums[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(v, sw, &tot);
    if (i < m) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *d_total = carry;
}

template <typename T>
__global__ void k_scan_add(T *out, size_t n, const T *sums) {
  size_t i = (size_t)blockIdx.x * kScanTile + threadIdx.x;
  T add = sums[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += add;
}

size_t scan_tmp_elems(size_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <typename T>
static wv_status scan_impl(const T *in, T *out, size_t n, T *total, T *tmp, cudaStream_t s) {
  if (n == 0) {
    WV_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    return WV_OK;
  }
  size_t tiles = (n + kScanTile - 1) / kScanTile;
  WV_LAUNCH("scan_tiles", k_scan_tiles<T>, (unsigned)tiles, kScanThreads, 0, s, in, out, n, tmp);
  WV_LAUNCH("scan_top", k_scan_top<T>, 1, kScanThreads, 0, s, tmp, tiles, total);
  if (tiles > 1)
    WV_LAUNCH("scan_add", k_scan_add<T>, (unsigned)tiles, kScanThreads, 0, s, out, n, (const T *)tmp);
  return WV_OK;
}
wv_status scan_exclusive_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total,
                             uint32_t *tmp, cudaStream_t s) {
  return scan_impl<uint32_t>(in, out, n, total, tmp, s);
}
wv_status scan_exclusive_u64(const uint64_t *in, uint64_t *out, size_t n, uint64_t *total,
                             uint64_t *tmp, cudaStream_t s) {
  return scan_impl<uint64_t>(in, out, n, total, tmp, s);
}

// The same scan launched without the profiler's bookkeeping (which keeps
// host-side tables and, when timing is on, creates events): used by the entry
// point that must not allocate anything.
wv_status scan_exclusive_u32_bare(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total,
                                  uint32_t *tmp, cudaStream_t s) {
  if (n == 0) {
    WV_CUDA(cudaMemsetAsync(total, 0, sizeof(uint32_t), s));
    return WV_OK;
  }
  const size_t tiles = (n + kScanTile - 1) / kScanTile;
  k_scan_tiles<uint32_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, tmp);
  k_scan_top<uint32_t><<<1, kScanThreads, 0, s>>>(tmp, tiles, total);
  if (tiles > 1) k_scan_add<uint32_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, tmp);
  WV_CUDA(cudaGetLastError());
  return WV_OK;
}

// ================================================================ options
wv_status resolve_config(const wv_options *opt, bool want_b, bool want_e, ResidueConfig *cfg) {
  ResidueConfig c;
  c.cong_b = want_b ? cong_default(0) : -2;
  c.cong_e = want_e ? cong_default(1) : -2;
  if (opt) {
    if (want_b && opt->cong_b >= 0) c.cong_b = opt->cong_b, c.cong_auto_b = false;
    if (want_e && opt->cong_e >= 0) c.cong_e = opt->cong_e, c.cong_auto_e = false;
    if (opt->block > 0) c.block = opt->block;
    if (opt->ilp > 0) c.ilp = c.ilp64 = opt->ilp;
    if (opt->tile_terms > 0) c.tile_terms = opt->tile_terms;
    if (opt->max_tiles > 0) c.max_tiles = opt->max_tiles;
    if (opt->tile_terms > 0 || opt->max_tiles > 0) c.tiles_auto = false;
    if (opt->blocks_per_sm > 0) c.blocks_per_sm = opt->blocks_per_sm;
    if (opt->arith > 0) c.arith = opt->arith;
    c.check_primes = opt->check_primes != 0;
    c.tiling = opt->tiling;
    if (opt->uform_min31 > 0) c.uform_min31 = (uint32_t)opt->uform_min31;
    if (opt->uform_min64 > 0) c.uform_min64 = (uint32_t)opt->uform_min64;
  }
  if (c.tiling < 0 || c.tiling > 2)
    return set_error(WV_EINVAL, "tiling=%d must be 0, 1 or 2", c.tiling);
  if (c.cong_b >= 0 && (c.cong_b >= cong_count() || cong_view(c.cong_b).kind != 0))
    return set_error(WV_EINVAL, "cong_b=%d is not a Bernoulli congruence", c.cong_b);
  if (c.cong_e >= 0 && (c.cong_e >= cong_count() || cong_view(c.cong_e).kind != 1))
    return set_error(WV_EINVAL, "cong_e=%d is not an Euler congruence", c.cong_e);
  if (c.block < 32 || c.block > 256 || c.block % 32)
    return set_error(WV_EINVAL, "block=%d must be a multiple of 32 in [32,256]", c.block);
  if (c.ilp != 1 && c.ilp != 2 && c.ilp != 4)
    return set_error(WV_EINVAL, "ilp=%d must be 1, 2 or 4", c.ilp);
  if (!arith_selectable(c.arith))
    return set_error(WV_EINVAL, "arith=%d is not a formulation of this library (%s)", c.arith,
                     kArithList);
  if (c.ilp == 4 && c.arith != 9 && !(c.arith >= 12 && c.arith <= 23))
    return set_error(WV_EINVAL, "ilp=4 is built for formulations 9 and 12..23 only (arith=%d)",
                     c.arith);
  if (c.arith >= 9) c.ilp64 = 1;  // the grouped 64-bit forms run one chain per thread
  if (c.max_tiles > 4096) return set_error(WV_EINVAL, "max_tiles=%d > 4096", c.max_tiles);
  *cfg = c;
  return WV_OK;
}

}  // namespace wv

// ================================================================ C ABI
using namespace wv;

extern "C" {

const char *wv_version(void) { return "wv 0.1 (sm_103a)"; }

int wv_is_prime(uint64_t n) {
  if (n >= WV_P_MAX) return -1;
  return wv::is_prime37(n) ? 1 : 0;
}
const char *wv_last_error(void) { return g_err.c_str(); }

int wv_congruence_count(void) { return cong_count(); }

wv_status wv_congruence_info(int id, int *kind, int *n_rows, int64_t *lhs, const char **name) {
  if (id < 0 || id >= cong_count()) return set_error(WV_EINVAL, "congruence id %d", id);
  const CongView &c = cong_view(id);
  if (kind) *kind = c.kind;
  if (n_rows) *n_rows = c.nrows;
  if (lhs) *lhs = c.lhs;
  if (name) *name = c.name;
  return WV_OK;
}

wv_status wv_congruence_row(int id, int row, int64_t *coef, uint32_t *xn, uint32_t *xd,
                            uint32_t *yn, uint32_t *yd) {
  if (id < 0 || id >= cong_count()) return set_error(WV_EINVAL, "congruence id %d", id);
  const CongView &c = cong_view(id);
  if (row < 0 || row >= c.nrows) return set_error(WV_EINVAL, "row %d of %s", row, c.name);
  const uint32_t *w = cong_row(c.row0 + (uint32_t)row);
  if (xn) *xn = w[0];
  if (xd) *xd = w[1];
  if (yn) *yn = w[2];
  if (yd) *yd = w[3];
  const bool plain = w[5] == 1 && cong_dist()[c.dist0 + cong_td()[w[4]]] == 1;
  if (coef) *coef = plain ? cong_tc()[w[4]] : 0;
  if (!plain) return set_error(WV_ERANGE, "row %d of %s has a coefficient sum c_k d_k^t", row, c.name);
  return WV_OK;
}

wv_status wv_congruence_terms(int id, int row, int64_t *c, uint64_t *d, int cap, int *n) {
  if (id < 0 || id >= cong_count()) return set_error(WV_EINVAL, "congruence id %d", id);
  const CongView &v = cong_view(id);
  if (row < 0 || row >= v.nrows) return set_error(WV_EINVAL, "row %d of %s", row, v.name);
  const uint32_t *w = cong_row(v.row0 + (uint32_t)row);
  if (n) *n = (int)w[5];
  for (uint32_t k = 0; k < w[5] && (int)k < cap; ++k) {
    if (c) c[k] = cong_tc()[w[4] + k];
    if (d) d[k] = cong_dist()[v.dist0 + cong_td()[w[4] + k]];
  }
  if ((int)w[5] > cap) return set_error(WV_ERANGE, "row has %u terms, capacity %d", w[5], cap);
  return WV_OK;
}

wv_status wv_general_row(int kind, int row, uint32_t *xn, uint32_t *xd, uint32_t *yn, uint32_t *yd,
                         int32_t c[3], uint32_t d[3], uint32_t lhs[3]) {
  if (kind < 0 || kind > 1) return set_error(WV_EINVAL, "kind %d", kind);
  const WvGenCongruence &g = kWvGeneral[kind];
  if (row < 0 || row >= g.nrows) return set_error(WV_EINVAL, "row %d of %s", row, g.name);
  const WvGenRow &r = g.rows[row];
  if (xn) *xn = r.xn;
  if (xd) *xd = r.xd;
  if (yn) *yn = r.yn;
  if (yd) *yd = r.yd;
  for (int i = 0; i < 3; ++i) {
    if (c) c[i] = r.c[i];
    if (d) d[i] = r.d[i];
    if (lhs) lhs[i] = g.lhs[i];
  }
  return WV_OK;
}

int wv_general_rows(int kind) { return (kind == 0 || kind == 1) ? kWvGeneral[kind].nrows : 0; }

wv_status wv_count_terms(const uint64_t *h_primes, size_t n, int cong_b, int cong_e,
                         uint64_t *terms_b, uint64_t *terms_e) {
  if (n && !h_primes) return set_error(WV_EINVAL, "h_primes is NULL");
  if (cong_b == -1 || cong_b < -2) cong_b = cong_default(0);
  if (cong_e == -1 || cong_e < -2) cong_e = cong_default(1);
  if (cong_b >= cong_count() || cong_e >= cong_count()) return set_error(WV_EINVAL, "bad congruence id");
  uint64_t tb = 0, te = 0;
  for (size_t i = 0; i < n; ++i) {
    uint64_t p = h_primes[i];
    if (p < 11 || p >= WV_P_MAX || (p & 1) == 0) continue;
    if (cong_b >= 0) {
      const CongView &c = cong_view(cong_b);
      for (int j = 0; j < c.nrows; ++j) tb += cong_row_terms(c.row0 + j, p);
    }
    if (cong_e >= 0) {
      const CongView &c = cong_view(cong_e);
      for (int j = 0; j < c.nrows; ++j) te += cong_row_terms(c.row0 + j, p);
    }
  }
  if (terms_b) *terms_b = tb;
  if (terms_e) *terms_e = te;
  return WV_OK;
}

void wv_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
}
void wv_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto &pe : g_pending) {
    g_event_pool.push_back(pe.a);
    g_event_pool.push_back(pe.b);
  }
  g_pending.clear();
  g_prof.clear();
  g_prof_names.clear();
  g_launches = 0;
}
wv_status wv_profile_collect(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto &pe : g_pending) {
    cudaError_t e = cudaEventSynchronize(pe.b);
    if (e != cudaSuccess) return cuda_fail(e, "wv_profile_collect");
    float ms = 0;
    cudaEventElapsedTime(&ms, pe.a, pe.b);
    g_prof[pe.name].total_ms += ms;
    g_event_pool.push_back(pe.a);
    g_event_pool.push_back(pe.b);
  }
  g_pending.clear();
  return WV_OK;
}
int wv_profile_kernels(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return (int)g_prof_names.size();
}
wv_status wv_profile_get(int idx, const char **name, uint64_t *launches, double *total_ms) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (idx < 0 || idx >= (int)g_prof_names.size()) return set_error(WV_EINVAL, "profile index");
  const std::string &nm = g_prof_names[idx];
  const ProfEntry &e = g_prof[nm];
  if (name) *name = nm.c_str();
  if (launches) *launches = e.launches;
  if (total_ms) *total_ms = e.total_ms;
  return WV_OK;
}
uint64_t wv_profile_launches(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_launches;
}

}  // extern "C"
