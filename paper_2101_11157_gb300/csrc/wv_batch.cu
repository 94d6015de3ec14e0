// wv_batch.cu -- step a8: many residue requests in one launch sequence.
//
// The primes of all requests are gathered into one array, planned together
// (one counting sort by p-bucket across every request), accumulated by one
// persistent work-stealing launch per arithmetic path with the largest
// primes first, finalised, and scattered back to each request's outputs.
// The whole sequence is captured once into a CUDA graph; wv_batch_run
// replays it.  This is the batched counterpart of calling wv_residues_pm3
// once per request.
#include <string.h>

#include <vector>

#include "../../include/wv_batch.h"
#include "wv_internal.h"

namespace wv {

struct ReqDesc {
  const uint64_t *primes;
  uint64_t *out_b, *out_e;
  uint64_t n, off;
};

__global__ void k_batch_gather(const ReqDesc *reqs, uint64_t *all) {
  const ReqDesc r = reqs[blockIdx.x];
  for (uint64_t i = threadIdx.x; i < r.n; i += blockDim.x) all[r.off + i] = r.primes[i];
}

__global__ void k_batch_scatter(const ReqDesc *reqs, const uint64_t *all_b, const uint64_t *all_e) {
  const ReqDesc r = reqs[blockIdx.x];
  for (uint64_t i = threadIdx.x; i < r.n; i += blockDim.x) {
    if (r.out_b) r.out_b[i] = all_b[r.off + i];
    if (r.out_e) r.out_e[i] = all_e[r.off + i];
  }
}

}  // namespace wv

using namespace wv;

struct wv_batch_s {
  int device = -1;
  size_t k = 0, n = 0;
  uint64_t *all = nullptr, *all_b = nullptr, *all_e = nullptr;
  ReqDesc *d_reqs = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_free(wv_batch_s *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
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
  cfg.chunk = n;  // one plan and one persistent launch per path for the whole batch
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));  // per-device set-up happens before the capture
  wv_batch_s *b = new wv_batch_s();
  b->device = dev->device;
  b->k = k;
  b->n = n;
  cudaError_t e = cudaMalloc(&b->all, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->all_b, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->all_e, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_reqs, k * sizeof(ReqDesc));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_reqs, table.data(), k * sizeof(ReqDesc), cudaMemcpyHostToDevice);
  // the replays run on the caller's stream, which need not be ordered after
  // a pageable copy: make sure it has landed
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "wv_batch_create");
  }
  // capture: gather -> plan/accumulate/finalise -> scatter
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  wv_status st = WV_OK;
  k_batch_gather<<<(unsigned)k, 256, 0, b->cap>>>(b->d_reqs, b->all);
  e = cudaGetLastError();
  if (e != cudaSuccess) st = cuda_fail(e, "batch gather");
  if (st == WV_OK) st = residues_device(b->all, n, b->all_b, b->all_e, cfg, b->cap);
  if (st == WV_OK) {
    k_batch_scatter<<<(unsigned)k, 256, 0, b->cap>>>(b->d_reqs, b->all_b, b->all_e);
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
