// wv_batch.cu -- step a8: many residue requests in one launch sequence.
//
// The primes of all requests are gathered into one array, grouped by the
// congruence pair that suits their size (the bands of the range-aware calls,
// chosen like the paper's own switch of congruence with p, Sec. 3), planned
// together per band (a counting sort by p-bucket across every request),
// accumulated by persistent work-stealing launches with the largest primes
// first, finalised, and scattered back to each request's outputs.  The bands
// run on forked streams inside one captured CUDA graph, so the tail of one
// band's launch overlaps the next; wv_batch_run replays the graph.  This is
// the batched counterpart of calling wv_residues_ex once per request (and
// per band).
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/wv_batch.h"
#include "wv_internal.h"

namespace wv {

struct ReqDesc {
  const uint64_t *primes;
  uint64_t *out_b, *out_e;
  uint64_t n, off;
};

// Gathered slot j holds prime map[j] = (request << 48) | index: the slots of
// one band are contiguous, bands in descending order of size.
constexpr int kMapShift = 48;

__global__ void k_batch_gather(const ReqDesc *reqs, const uint64_t *map, uint64_t n, uint64_t *all) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint64_t m = map[j];
  all[j] = reqs[m >> kMapShift].primes[m & ((1ull << kMapShift) - 1)];
}

__global__ void k_batch_scatter(const ReqDesc *reqs, const uint64_t *map, uint64_t n,
                                const uint64_t *all_b, const uint64_t *all_e) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint64_t m = map[j];
  const ReqDesc r = reqs[m >> kMapShift];
  const uint64_t i = m & ((1ull << kMapShift) - 1);
  if (r.out_b) r.out_b[i] = all_b[j];
  if (r.out_e) r.out_e[i] = all_e[j];
}

}  // namespace wv

using namespace wv;

struct wv_batch_s {
  int device = -1;
  size_t k = 0, n = 0;
  uint64_t *all = nullptr, *all_b = nullptr, *all_e = nullptr;
  uint64_t *d_map = nullptr;
  ReqDesc *d_reqs = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> fork;  // one stream per band (capture only)
  std::vector<cudaEvent_t> ev;     // fork/join events (capture only)
  int bands = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_free(wv_batch_s *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaStream_t f : b->fork) cudaStreamDestroy(f);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  cudaFree(b->d_map);
  cudaFree(b->all);
  cudaFree(b->all_b);
  cudaFree(b->all_e);
  cudaFree(b->d_reqs);
  delete b;
}

extern "C" {

wv_status wv_batch_create(const wv_request *reqs, size_t k, const wv_options *opt, wv_batch *out) {
  clear_error();
  if (!out) return set_error(WV_EINVAL, "out is NULL");
  *out = nullptr;
  if (k == 0 || !reqs) return set_error(WV_EINVAL, "no requests");
  if (k > 65535) return set_error(WV_EINVAL, "at most 65535 requests per batch");
  std::vector<ReqDesc> table(k);
  size_t n = 0;
  for (size_t i = 0; i < k; ++i) {
    if (reqs[i].n && !reqs[i].d_primes) return set_error(WV_EINVAL, "request %zu: d_primes is NULL", i);
    if (reqs[i].n >= (1ull << kMapShift)) return set_error(WV_EINVAL, "request %zu is too long", i);
    table[i].primes = reqs[i].d_primes;
    table[i].out_b = reqs[i].d_out_b;
    table[i].out_e = reqs[i].d_out_e;
    table[i].n = reqs[i].n;
    table[i].off = n;
    n += reqs[i].n;
  }
  if (n == 0) return set_error(WV_EINVAL, "all requests are empty");
  ResidueConfig cfg;
  WV_CHECK(resolve_config(opt, true, true, &cfg));
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));  // per-device set-up happens before the capture

  // Group the slots by congruence pair: read the primes once, pick each
  // prime's pair as the range-aware calls would for [p, p + 1), and keep a
  // pair fixed where the caller chose it.  Groups are ordered by their work
  // (sum of p, largest first); inside a group, requests stay in order.
  struct Slot {
    int group;
    uint64_t key;
  };
  std::vector<Slot> slots;
  slots.reserve(n);
  std::vector<std::pair<int, int>> pairs;  // group -> (cong_b, cong_e)
  std::vector<double> work;
  {
    // the primes must be in place: wait for every stream's work first
    WV_CUDA(cudaDeviceSynchronize());
    std::vector<uint64_t> h;
    for (size_t r = 0; r < k; ++r) {
      h.resize(reqs[r].n);
      if (reqs[r].n)
        WV_CUDA(cudaMemcpy(h.data(), reqs[r].d_primes, reqs[r].n * 8, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < reqs[r].n; ++i) {
        int cb = cfg.cong_b, ce = cfg.cong_e;
        if (cfg.cong_auto_b || cfg.cong_auto_e) {
          int rb = 0, re = 0;
          cong_for_range(h[i] < ~0ull ? h[i] + 1 : h[i], &rb, &re);
          if (cfg.cong_auto_b) cb = rb;
          if (cfg.cong_auto_e) ce = re;
        }
        int g = 0;
        while (g < (int)pairs.size() && pairs[g] != std::make_pair(cb, ce)) ++g;
        if (g == (int)pairs.size()) {
          pairs.emplace_back(cb, ce);
          work.push_back(0.0);
        }
        work[g] += (double)h[i];
        slots.push_back({g, ((uint64_t)r << kMapShift) | (uint64_t)i});
      }
    }
  }
  std::vector<int> order(pairs.size());
  for (size_t g = 0; g < order.size(); ++g) order[g] = (int)g;
  std::sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
  std::vector<int> rank(pairs.size());
  for (size_t i = 0; i < order.size(); ++i) rank[order[i]] = (int)i;
  std::stable_sort(slots.begin(), slots.end(),
                   [&](const Slot &a, const Slot &c) { return rank[a.group] < rank[c.group]; });
  std::vector<uint64_t> map(n);
  std::vector<size_t> g_off(order.size() + 1, 0);
  for (size_t j = 0; j < n; ++j) {
    map[j] = slots[j].key;
    ++g_off[rank[slots[j].group] + 1];
  }
  for (size_t g = 0; g < order.size(); ++g) g_off[g + 1] += g_off[g];

  wv_batch_s *b = new wv_batch_s();
  b->device = dev->device;
  b->k = k;
  b->n = n;
  b->bands = (int)order.size();
  cudaError_t e = cudaMalloc(&b->all, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->all_b, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->all_e, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_map, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_reqs, k * sizeof(ReqDesc));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_reqs, table.data(), k * sizeof(ReqDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_map, map.data(), n * 8, cudaMemcpyHostToDevice);
  // the replays run on the caller's stream, which need not be ordered after
  // a pageable copy: make sure it has landed
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int g = 0; e == cudaSuccess && g <= b->bands; ++g) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev.push_back(ev);
    if (e == cudaSuccess && g < b->bands) {
      cudaStream_t f = nullptr;
      e = cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->fork.push_back(f);
    }
  }
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "wv_batch_create");
  }
  // capture: gather -> per group on its own stream: plan/accumulate/finalise
  // -> join -> scatter
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  wv_status st = WV_OK;
  const unsigned gb = (unsigned)((n + 255) / 256);
  k_batch_gather<<<gb, 256, 0, b->cap>>>(b->d_reqs, b->d_map, n, b->all);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(b->ev[b->bands], b->cap);
  if (e != cudaSuccess) st = cuda_fail(e, "batch gather");
  for (int g = 0; st == WV_OK && g < b->bands; ++g) {
    cudaStream_t f = b->fork[g];
    e = cudaStreamWaitEvent(f, b->ev[b->bands], 0);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "batch fork");
      break;
    }
    ResidueConfig c = cfg;
    c.cong_b = pairs[order[g]].first;
    c.cong_e = pairs[order[g]].second;
    const size_t o = g_off[g], m = g_off[g + 1] - g_off[g];
    c.chunk = m;  // one plan and one persistent launch per path for the group
    st = residues_device(b->all + o, m, b->all_b + o, b->all_e + o, c, f);
    if (st != WV_OK) break;
    e = cudaEventRecord(b->ev[g], f);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev[g], 0);
    if (e != cudaSuccess) st = cuda_fail(e, "batch join");
  }
  if (st == WV_OK) {
    k_batch_scatter<<<gb, 256, 0, b->cap>>>(b->d_reqs, b->d_map, n, b->all_b, b->all_e);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "batch scatter");
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap, &g);
  if (st == WV_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
  b->graph = g;
  if (st == WV_OK) {
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
  }
  if (st != WV_OK) {
    cudaGetLastError();
    batch_free(b);
    return st;
  }
  *out = b;
  return WV_OK;
}

wv_status wv_batch_run(wv_batch b, wv_stream stream) {
  clear_error();
  if (!b || !b->exec) return set_error(WV_EINVAL, "invalid batch handle");
  int dev = -1;
  WV_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) return set_error(WV_EINVAL, "batch belongs to device %d, current is %d",
                                         b->device, dev);
  prof_begin("batch_graph", (cudaStream_t)stream);
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  prof_end("batch_graph", (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return WV_OK;
}

wv_status wv_batch_info(wv_batch b, size_t *n_requests, size_t *n_primes, size_t *graph_nodes) {
  clear_error();
  if (!b) return set_error(WV_EINVAL, "invalid batch handle");
  if (n_requests) *n_requests = b->k;
  if (n_primes) *n_primes = b->n;
  if (graph_nodes) {
    size_t nn = 0;
    WV_CUDA(cudaGraphGetNodes(b->graph, nullptr, &nn));
    *graph_nodes = nn;
  }
  return WV_OK;
}

wv_status wv_batch_groups(wv_batch b, size_t *n_groups) {
  clear_error();
  if (!b) return set_error(WV_EINVAL, "invalid batch handle");
  if (n_groups) *n_groups = (size_t)b->bands;
  return WV_OK;
}

wv_status wv_batch_destroy(wv_batch b) {
  clear_error();
  if (!b) return WV_OK;
  const int bdev = b->device;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != bdev) cudaSetDevice(bdev);
  cudaError_t e = cudaDeviceSynchronize();
  batch_free(b);
  if (cur != bdev && cur >= 0) cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_fail(e, "wv_batch_destroy");
  return WV_OK;
}

}  // extern "C"
