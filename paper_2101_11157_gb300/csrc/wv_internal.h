// wv_internal.h -- host-side runtime shared by the library's translation units:
// error reporting, per-device state, stream-ordered scratch, launch profiling,
// and the device-wide scan used by the sieve and the planner.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

#include "../../include/wv.h"

namespace wv {

// ------------------------------------------------------------ errors
wv_status set_error(wv_status st, const char *fmt, ...);
void clear_error();
wv_status cuda_fail(cudaError_t e, const char *where);

#define WV_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return ::wv::cuda_fail(_e, #call);           \
  } while (0)

#define WV_CHECK(expr)                                                  \
  do {                                                                  \
    wv_status _s = (expr);                                              \
    if (_s != WV_OK) return _s;                                         \
  } while (0)

// ------------------------------------------------------------ device state
struct DeviceState {
  int device = -1;
  int sms = 0;
  int cc_major = 0, cc_minor = 0;
  cudaMemPool_t pool = nullptr;
  uint32_t *base_primes = nullptr;  // odd primes 3 .. sqrt(WV_P_MAX), device
  uint32_t n_base = 0;
  // the congruence registry (wv_registry.cu), device copy
  uint32_t *cg_rows = nullptr;
  int64_t *cg_tc = nullptr;
  uint16_t *cg_td = nullptr;
  uint64_t *cg_dist = nullptr;
};
// State of the current device, created on first use.
wv_status device_state(DeviceState **out);

// ------------------------------------------------------------ congruences
// Every runnable congruence (wv_registry.cu): ids 0 .. cong_count()-1 are the
// built-in and generated ones (selectable through wv_options); the general-
// index forms follow at cong_general_id(kind).  Row r of the registry is
// (sum_k c_k d_k^t) S_t(xn/xd, yn/yd): words xn, xd, yn, yd, first term,
// number of terms; term k is (cong_tc()[k], index cong_td()[k] into the
// congruence's distinct bases cong_dist()[dist0 ..]).
struct CongView {
  const char *name;
  int kind;       // 0 = Bernoulli, 1 = Euler
  int nrows;
  int64_t lhs;    // the left side (0 for the general-index forms)
  uint32_t row0, dist0, ndist;
};
int cong_count();
int cong_default(int kind);
void cong_for_range(uint64_t hi, int *cb, int *ce);
int cong_general_id(int kind);
const CongView &cong_view(int id);
const uint32_t *cong_row(uint32_t r);
const int64_t *cong_tc();
const uint16_t *cong_td();
const uint64_t *cong_dist();
uint64_t cong_row_terms(uint32_t r, uint64_t p);  // terms of row r for prime p
wv_status cong_upload(DeviceState *d);

// ------------------------------------------------------------ scratch
// Stream-ordered allocation from the library's own memory pool.
wv_status scratch_alloc(void **ptr, size_t bytes, cudaStream_t s);
void scratch_free(void *ptr, cudaStream_t s);

// RAII list of scratch blocks freed (stream-ordered) on scope exit.
struct Scratch {
  cudaStream_t s;
  void *ptrs[32];
  int n = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (int i = n - 1; i >= 0; --i) scratch_free(ptrs[i], s);
  }
  template <typename T>
  wv_status get(T **p, size_t count) {
    void *v = nullptr;
    wv_status st = scratch_alloc(&v, count * sizeof(T) + 256, s);
    if (st != WV_OK) return st;
    ptrs[n++] = v;
    *p = reinterpret_cast<T *>(v);
    return WV_OK;
  }
};

// ------------------------------------------------------------ profiling
void prof_begin(const char *name, cudaStream_t s);
void prof_end(const char *name, cudaStream_t s);

#define WV_LAUNCH(name, kern, grid, block, smem, stream, ...)           \
  do {                                                                  \
    ::wv::prof_begin(name, stream);                                     \
    kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);           \
    ::wv::prof_end(name, stream);                                       \
    cudaError_t _le = cudaGetLastError();                               \
    if (_le != cudaSuccess) return ::wv::cuda_fail(_le, name);          \
  } while (0)

// ------------------------------------------------------------ scan
// Exclusive prefix sum of n values; *d_total (device) receives the sum.
// tmp must hold scan_tmp_elems(n) elements.
size_t scan_tmp_elems(size_t n);
wv_status scan_exclusive_u32(const uint32_t *d_in, uint32_t *d_out, size_t n,
                             uint32_t *d_total, uint32_t *d_tmp, cudaStream_t s);
wv_status scan_exclusive_u64(const uint64_t *d_in, uint64_t *d_out, size_t n,
                             uint64_t *d_total, uint64_t *d_tmp, cudaStream_t s);
wv_status scan_exclusive_u32_bare(const uint32_t *d_in, uint32_t *d_out, size_t n,
                                  uint32_t *d_total, uint32_t *d_tmp, cudaStream_t s);

// ------------------------------------------------------------ residues
struct ResidueConfig {
  int cong_b = 6;        // set by resolve_config (cong_default); -2 = skip
  int cong_e = 12;       // set by resolve_config (cong_default); -2 = skip
  bool cong_auto_b = true;  // not chosen by the caller: range-aware calls pick by p
  bool cong_auto_e = true;
  int block = 256;
  int ilp = 1;            // chains per thread, p < 2^31
  int ilp64 = 1;          // chains per thread, 2^31 <= p < 2^37
  int tile_terms = 1 << 20;
  int max_tiles = 8;
  bool tiles_auto = true; // few primes: more, shorter tiles (see tile_shape)
  int blocks_per_sm = 0;  // 0 = occupancy
  int arith = 50;         // hot-loop formulation (see wv_accum.cuh)
  uint32_t gen_e_b = 0;   // general index: B_{p-e} (e odd); 0 = the B_{p-3} forms
  uint32_t gen_e_e = 0;   // general index: E_{p-1-e} (e even); 0 = the E_{p-3} forms
  size_t chunk = 0;       // primes per launch sequence (0: library default 16384)
  bool check_primes = false;  // planner verifies primality (composites -> invalid slot)
  int tiling = 0;         // 0 / 2: lane chains where supported, 1: warp tiles
  uint32_t uform_min31 = 3072, uform_min64 = 32768;  // u form from pieces this long (48..50)
  uint64_t epoch_piece_max = 1ull << 17;  // longest lane chain of a serving plan
  // lane chains apply to the grouped formulations 50 (the default), 31, 39
  // and the lane-only forms 40..49, with ILP 1 or 2, and not to the general
  // index (its own single-term tiles)
  bool lane_chains() const {
    return tiling != 1 && (arith == 31 || arith >= 39) && (ilp == 1 || ilp == 2) && !gen_e_b &&
           !gen_e_e;
  }
};
wv_status resolve_config(const wv_options *opt, bool want_b, bool want_e, ResidueConfig *cfg);

// The hot-loop formulations a caller may select (wv_options.arith):
//   32-bit path (p < 2^31): 1, 2, 4 single terms; 9 groups of 2 cubes / 3
//   squares; 25..28 form 9 with other ALU/multiply-pipe splits of the table
//   additions; 29, 30, 31 groups of 3 cubes, 4 squares, or both; 39 groups
//   of 4 cubes / 5 squares; with lane chains also 40 (5 / 6), 41 (4 / 6) and
//   44 (4 / 7), the u forms 45 (8 / 10), 46 (6 / 8), 47 (10 / 12), and 48,
//   49, 50 (the default: per warp 45 on long pieces, 41 on short ones)
//   (M31Form in wv_accum.cuh).
//   64-bit path (2^31 <= p < 2^37): 1, 2, 4 single terms; every
//   other value runs the grouped default (8 cubes / 12 squares) except 12..18
//   and 21, other group sizes and register budgets, 32..36, the default
//   with its table additions as PTX carry chains, 37, the default with the
//   earlier, longer shrink of its tables, and 38, the default with its
//   per-chain set-up unrolled as it was; with lane chains 42, 43 (10 or 11
//   squares), 49 (the u form, 12 cubes / 16 squares) and 50 (the default:
//   per warp 49 on long pieces, the grouped form below).  23: the paper's own
//   arithmetic on both paths.
constexpr const char *kArithList = "1, 2, 4, 9, 12..18, 21, 23, 25..52";
inline bool arith_selectable(int a) {
  return a == 1 || a == 2 || a == 4 || a == 9 || (a >= 12 && a <= 18) || a == 21 || a == 23 ||
         (a >= 25 && a <= 52);
}

// Residues for n primes (device array), asynchronous on s.
wv_status residues_device(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                          uint64_t *d_out_e, const ResidueConfig &cfg, cudaStream_t s);

// ---- phases of one residue computation, for the serving loop
struct Plan;  // device-side plan of one prime list (wv_residue.cu)
struct EpochItem {
  uint32_t plan;    // index into the epoch's plan array
  uint32_t first;   // first tile of the item's range
  uint32_t count;   // tiles in the range
  uint32_t prefix;  // tiles of all earlier items
};
struct PlanState {
  Plan *host = nullptr;     // host copy of the plan (device pointers inside)
  void *blocks[16] = {};
  int nblocks = 0;
  size_t bytes = 0;         // device bytes held
  uint32_t n = 0, total = 0, split = 0;  // primes, tiles, first 64-bit tile
  double terms[2] = {-1, -1};  // with lane chains: terms on the 32-bit / 64-bit kernel
};
// Allocate (stream-ordered) and plan n <= 65536 primes; asynchronous.  With
// lane chains and `terms` (upper bounds on the plan's terms on the 32-bit and
// the 64-bit kernel), the chain lengths are fixed on the host and bounded
// for epochs; without, they follow the device's term counts.
wv_status plan_build(const uint64_t *d_primes, uint32_t n, const ResidueConfig &cfg,
                     PlanState *ps, cudaStream_t s, const double *terms = nullptr);
// Device bytes plan_build will hold for n primes (the same `terms`).
size_t plan_bytes(uint32_t n, const ResidueConfig &cfg, const double *terms = nullptr);
// Synchronise s and read the plan's tile totals (and, with lane chains, its
// exact terms per kernel) into ps.
wv_status plan_totals(PlanState *ps, cudaStream_t s);
// Copy the plan struct to device memory at d_plan (asynchronous).
wv_status plan_upload(const PlanState *ps, Plan *d_plan, cudaStream_t s);
size_t plan_struct_bytes();
// Epoch launch over items (device array) of plans (device array).
wv_status epoch_launch(bool wide, const EpochItem *d_items, uint32_t n_items, uint32_t total,
                       const Plan *d_plans, uint32_t *d_counter, const ResidueConfig &cfg,
                       int sms,
                       int reserve_blocks, cudaStream_t s);
// One launch for items of both paths (bit 31 of EpochItem::plan marks 64-bit items).
// `reserve_blocks` leaves room on the SMs for concurrent kernels of other streams.
wv_status epoch_launch_mixed(const EpochItem *d_items, uint32_t n_items, uint32_t total,
                             const Plan *d_plans, uint32_t *d_counter, const ResidueConfig &cfg,
                             int sms, int reserve_blocks, cudaStream_t s);
// Non-persistent form: one warp per tile (grid = total tiles), no counter.
wv_status epoch_launch_tiles(const EpochItem *d_items, uint32_t n_items, uint32_t total,
                             const Plan *d_plans, const ResidueConfig &cfg, cudaStream_t s);
// Finalise every prime of the plan into d_out_b / d_out_e (asynchronous).
wv_status plan_finalize(PlanState *ps, uint64_t *d_out_b, uint64_t *d_out_e, cudaStream_t s);
void plan_free(PlanState *ps, cudaStream_t s);

// Sieve primitives
wv_status sieve_device(uint64_t lo, uint64_t hi, uint64_t *d_out, size_t cap,
                       uint64_t *count_host, cudaStream_t s);

}  // namespace wv
