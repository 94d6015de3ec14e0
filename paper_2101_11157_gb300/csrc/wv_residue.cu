// wv_residue.cu -- steps a2-a6: plan, term generation, accumulation, reduction
// and finalisation of B_{p-3} mod p and E_{p-3} mod p.
//
// Method (Sec. 3, "It remains to describe how to calculate these sums"; Sec. 5
// after eqn 5.6): every congruence row contributes coef * S(x, y) with
// S = sum_{xp<s<yp} s^-e (e = 3 for B_{p-3}, e = 2 for E_{p-3}).  S is the
// ratio c1/c0 of the two lowest coefficients of prod (z + s^e), built one
// term at a time by eqn 3.12 (c1 <- c1 t + c0, c0 <- c0 t, t = s^e); pieces
// of a product are merged with eqn 3.14.  One modular inverse per prime
// finishes the sum (Sec. 3, the CPU's last step in the paper's GPU method).
//
// GB300 design:
//  * Work unit (default) = a lane chain: one lane's contiguous range of s
//    inside one (prime, row) sum.  The planner splits every sum into pieces
//    of at most L terms (L: the path's terms over 16 times its resident
//    lanes, at least 4096 / 16384), sorts the pieces by class and length,
//    and a persistent kernel (grid = SMs x occupancy) lets warps take 32
//    pieces at a time from an atomic counter, longest first.  The lanes of a
//    warp then sum different primes and rows side by side, and a sum of any
//    length keeps one chain per piece, so the per-chain set-up stays small
//    even for the thousands of short sums of the generated congruences.
//  * Work unit (wv_options.tiling = 1) = a warp tile: a contiguous range of s
//    inside one sum, split over the 32 lanes x ILP chains of a warp and merged
//    by shuffles.  The planner splits every sum into at most `max_tiles`
//    tiles of about `tile_terms` terms, taken largest primes first.
//  * Inside a piece, each lane owns ILP contiguous runs of s.  Term
//    generation is by forward differences (Sec. 3, improvement 1): s^3 from
//    (s-1)^3 with three modular additions, s^2 with one; no multiplication.
//  * Accumulation: signed Montgomery arithmetic (see wv_arith.cuh).  For
//    p < 2^30 a term costs 7 integer multiplies (hi(c0 t), hi(c1 t), t p^-1,
//    c0 tq, c1 tq, hi(m0 p), hi(m1 p)); 64-bit words for 2^30 <= p < 2^37.
//  * The chains of a lane are merged with eqn 3.14 in registers (of a warp
//    tile, also by warp shuffles); one (c0, c1) pair per tile goes to global
//    memory.  The finalise
//    kernel (one warp per prime and kind) merges the tiles of each sum, forms
//    sum_j coef_j c1_j / c0_j as one fraction, and inverts once (Fermat).
//
// Montgomery bookkeeping: the hot step multiplies by a plain t with REDC, so
// c0 and c1 drift by powers of R, but the ratio c1/c0 always equals S * R
// (true initially for (c0, c1) = (R, 0) and preserved by both eqn 3.12 steps
// and by eqn 3.14 under REDC).  The finaliser therefore divides by R once.
#include "wv_prime.cuh"
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "wv_accum.cuh"

namespace wv {

// ------------------------------------------------------------------ planner
// Primes are ordered into slots by p-bucket floor(log2 p), ascending (a
// counting sort; order inside a bucket is arbitrary and does not affect any
// result).  Buckets 0..30 are the p < 2^31 slots of the 32-bit kernel; the
// accumulation kernels walk slots from the top, so the largest primes start
// first.
__device__ __forceinline__ uint32_t p_bucket(uint64_t p) {
  const bool valid = (p >= 11) && (p & 1) && (p < kPMax);
  return valid ? (uint32_t)(63 - __clzll((long long)p)) : 0u;  // special/invalid: no sums
}

__global__ void k_plan_prime(Plan P) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const uint32_t b = p_bucket(P.primes[i]);
  P.flag[i] = b;
  atomicAdd(&P.bk[b], 1u);
}

__global__ void k_plan_buckets(Plan P) {  // one warp: offsets of the 64 buckets
  const int lane = threadIdx.x;
  uint32_t c0 = P.bk[lane], c1 = P.bk[32 + lane];
  uint32_t x0 = c0, x1 = c1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
    if (lane >= o) { x0 += y0; x1 += y1; }
  }
  const uint32_t tot0 = __shfl_sync(0xffffffffu, x0, 31);
  P.bk[64 + lane] = x0 - c0;
  P.bk[96 + lane] = tot0 + x1 - c1;
  // buckets 0..30 (p < 2^31) go to the 32-bit kernel: signed words below
  // 2^30, unsigned words from 2^30 to 2^31
  const uint32_t below31 = __shfl_sync(0xffffffffu, x0, 30);
  if (lane == 0) *P.n31 = below31;
}

__global__ void k_plan_scatter(Plan P) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  uint64_t p = P.primes[i];
  const uint32_t b = P.flag[i];
  const uint32_t slot = P.bk[64 + b] + atomicAdd(&P.bk[128 + b], 1u);
  PrimeCtx c;
  bool valid = (p >= 5) && (p & 1) && (p < kPMax);
  if (valid && P.check) valid = is_prime37(p);
  if (valid && p >= 11) {
    c = make_ctx(p, i);
  } else {
    c.p = p; c.q = 0; c.one = 0; c.r2 = 0; c.orig = i;
    c.flags = 2u | ((p >= kM31Limit) ? 1u : 0u);  // no sums: special or invalid
  }
  P.ctx[slot] = c;
}

__global__ void k_plan_segments(Plan P) {
  uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.n * P.rows_pp) return;
  uint32_t slot = idx / P.rows_pp, j = idx - slot * P.rows_pp;
  const PrimeCtx c = P.ctx[slot];
  uint64_t lo = 0, cnt = 0;
  uint32_t tiles = 0;
  if (!(c.flags & 2u)) {
    const uint64_t p = c.p;
    // open interval (x p, y p): s = floor(xn p / xd) + 1 .. floor(yn p / yd)
    // (registry endpoints are 32-bit words with x, y <= 1/2)
    const uint32_t *w = P.cg_rows + 6 * (size_t)(j < P.rows_b ? P.rb0 + j : P.re0 + (j - P.rows_b));
    lo = floor_frac_times(w[0], w[1], p) + 1;
    uint64_t hi = floor_frac_times(w[2], w[3], p) + 1;
    cnt = hi > lo ? hi - lo : 0;
    if (cnt) {
      uint64_t t = (cnt + P.tile_terms - 1) / P.tile_terms;
      tiles = (uint32_t)(t < 1 ? 1 : (t > P.max_tiles ? P.max_tiles : t));
    }
  }
  P.seg_lo[idx] = lo;
  P.seg_cnt[idx] = cnt;
  P.seg_tiles[idx] = tiles;
}

// tile -> segment map: every segment writes its index into its tiles' slots
__global__ void k_plan_tilemap(Plan P) {
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.n * P.rows_pp) return;
  const uint32_t f = P.seg_first[idx], T = P.seg_tiles[idx];
  for (uint32_t t = 0; t < T; ++t) P.tile_seg[f + t] = idx;
}

__global__ void k_plan_split(Plan P) {
  uint32_t n31 = *P.n31;
  *P.split_tile = (n31 < P.n) ? P.seg_first[n31 * P.rows_pp] : *P.total_tiles;
  P.counters[0] = 0;
  P.counters[1] = 0;
}

// ------------------------------------------------------------------ lane chains
// With lane chains every tile is one lane's piece of a segment.  The planner
// splits segment s into ceil(cnt_s / L) pieces, where the chain length L of
// the segment's path (32-bit or 64-bit kernel) is the larger of a floor that
// keeps the per-chain set-up small and the path's terms over the number of
// chains that fill the GPU kLaneRounds times over (so that no chain runs
// longer than about 1/kLaneRounds of the launch, and the longest start
// first); it then
// sorts the tiles by class (signed 32-bit, unsigned 32-bit, 64-bit; B or E)
// and, inside a class, by length (32 steps per octave), so that the
// lanes of a warp run one code path for about the same number of terms.
constexpr int kChainClasses = 6;
constexpr uint32_t kChainBins = 2048;  // length bins per class
// chains wanted per path: resident threads per SM (3 blocks of 256 on the
// 32-bit kernel, 2 on the 64-bit one) x SMs x rounds (kLaneRounds for a
// call, kLaneRoundsEpoch for a serving plan, whose epochs mix many plans);
// shortest chain lengths (the 64-bit path's set-up costs about 40 groups)
constexpr uint64_t kLaneThreads31 = 768, kLaneThreads64 = 512;
constexpr uint64_t kLaneRounds = 16, kLaneRoundsEpoch = 4;
// a serving plan's chains are at most ResidueConfig::epoch_piece_max terms
// long (2^17 by default), so that an epoch is never held up long by one chain
// (2^17 terms are about 8 ms of one lane on the 32-bit kernel, 13 ms on the
// 64-bit one) and the shortest epochs still hold enough warps to fill the GPU;
// shorter caps pay more per-chain set-ups (2^16 served a mixed stream 2 %
// slower), longer ones let single chains hold epochs (2^20: 2 % slower)
constexpr uint64_t kLaneMin31 = 4096, kLaneMin64 = 16384;

__global__ void k_lane_sum(Plan P) {  // terms per path: one atomic per block and path
  __shared__ unsigned long long sh[2][8];
  const size_t ns = (size_t)P.n * P.rows_pp, stride = (size_t)gridDim.x * blockDim.x;
  const uint32_t n31 = *P.n31;
  uint64_t c31 = 0, c64 = 0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < ns; idx += stride) {
    const uint64_t c = P.seg_cnt[idx];
    if (idx / P.rows_pp >= n31) c64 += c; else c31 += c;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    c31 += __shfl_down_sync(0xffffffffu, c31, o);
    c64 += __shfl_down_sync(0xffffffffu, c64, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[0][w] = c31, sh[1][w] = c64;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += sh[0][i], b += sh[1][i];
    if (a) atomicAdd((unsigned long long *)&P.lane_sum[0], a);
    if (b) atomicAdd((unsigned long long *)&P.lane_sum[1], b);
  }
}

__device__ __forceinline__ uint64_t lane_chain_len(const Plan &P, int path) {
  const uint64_t t = P.lane_target[path];
  const uint64_t L = (P.lane_sum[path] + t - 1) / t;
  return L > P.lane_min[path] ? L : P.lane_min[path];
}

__global__ void k_lane_chains(Plan P) {  // pieces per segment
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)P.n * P.rows_pp) return;
  const uint64_t cnt = P.seg_cnt[idx];
  uint32_t t = 0;
  if (cnt) {
    const int path = idx / P.rows_pp >= *P.n31 ? 1 : 0;
    const uint64_t L = P.lane_fix[path] ? P.lane_fix[path] : lane_chain_len(P, path);
    t = (uint32_t)((cnt + L - 1) / L);  // <= terms / L + 1: within the tile capacity
  }
  P.seg_tiles[idx] = t;
}


// Sort key of the T pieces of segment s: class * kChainBins + length bin of
// the longest piece (the others are one term shorter at most).  The kernels
// take warps from the top of their range, so the longest pieces start first.
__device__ __forceinline__ uint32_t seg_key(const Plan &P, uint32_t s, uint32_t T) {
  const uint32_t slot = s / P.rows_pp, j = s - slot * P.rows_pp;
  const uint64_t cnt = P.seg_cnt[s];
  const uint64_t n = (cnt + T - 1) / T;  // >= 1
  const uint32_t path = slot >= *P.n31 ? 2u : (P.ctx[slot].flags & 1u) ? 1u : 0u;
  const uint32_t cls = path * 2 + (j >= P.rows_b ? 1u : 0u);
  const uint32_t e = 63 - __clzll((long long)n);
  const uint32_t frac = (uint32_t)((e >= 5 ? n >> (e - 5) : n << (5 - e)) & 31u);
  return cls * kChainBins + (e * 32 + frac);
}

// The histogram and scatter kernels visit the segments in tiles of kTileRows
// rows by 32 primes: the block's threads load the tile prime by prime (a
// prime's rows are contiguous, so a sector serves 8 rows), stage it in
// shared memory, and each warp then takes one row of the tile across its 32
// primes: neighbouring primes' pieces of one row mostly share a length bin,
// so that one atomic serves the warp.
constexpr uint32_t kTileRows = 8, kTileThreads = 32 * kTileRows;
struct TileIdx {
  uint32_t slot, j;  // the thread's (prime, row) in the load phase
  bool ok;
};
__device__ __forceinline__ TileIdx tile_load_idx(const Plan &P, size_t tile) {
  const size_t nst = (P.n + 31) / 32;
  const uint32_t j0 = (uint32_t)(tile / nst) * kTileRows, slot0 = (uint32_t)(tile % nst) * 32;
  TileIdx r;
  r.slot = slot0 + (threadIdx.x / kTileRows);
  r.j = j0 + (threadIdx.x % kTileRows);
  r.ok = r.slot < P.n && r.j < P.rows_pp;
  return r;
}
__device__ __forceinline__ size_t tile_count(const Plan &P) {
  return (size_t)((P.rows_pp + kTileRows - 1) / kTileRows) * ((P.n + 31) / 32);
}

// counts per key: segments of one piece add through one atomic per key and
// warp, longer segments their piece count each; keys kept for the scatter
__global__ void __launch_bounds__(kTileThreads) k_chain_hist(Plan P) {
  __shared__ uint32_t shT[kTileRows][33], shK[kTileRows][33];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t nt = tile_count(P);
  for (size_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const TileIdx ti = tile_load_idx(P, tile);
    uint32_t T = 0, key = 0;
    if (ti.ok) {
      const uint32_t s = ti.slot * P.rows_pp + ti.j;
      T = P.seg_tiles[s];
      if (T) {
        key = seg_key(P, s, T);
        P.chain_key[s] = key;
      }
    }
    shT[threadIdx.x % kTileRows][threadIdx.x / kTileRows] = T;
    shK[threadIdx.x % kTileRows][threadIdx.x / kTileRows] = key;
    __syncthreads();
    T = shT[w][lane];
    key = shK[w][lane];
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xffffffffu, T == 1 ? key : 0xffff0000u | lane);
    if (T == 1 && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&P.chain_hist[key], (uint32_t)__popc(peers));
    if (T > 1) atomicAdd(&P.chain_hist[key], T);
  }
}

// one block: counts -> first positions, each class starting on a whole warp;
// padding slots get kNoChain; lane_w = {32-bit kernel's warps, all warps}
constexpr int kOffThreads = 1024;
__global__ void __launch_bounds__(kOffThreads) k_chain_offsets(Plan P) {
  __shared__ uint32_t sh[kOffThreads];
  __shared__ uint32_t base;
  const uint32_t t = threadIdx.x;
  constexpr uint32_t per = kChainBins / kOffThreads;  // bins per thread and class
  if (t == 0) base = 0;
  __syncthreads();
  for (int c = 0; c < kChainClasses; ++c) {
    uint32_t h[per], v = 0;
#pragma unroll
    for (uint32_t i = 0; i < per; ++i) {
      h[i] = P.chain_hist[c * kChainBins + t * per + i];
      v += h[i];
    }
    sh[t] = v;
    __syncthreads();
    for (uint32_t o = 1; o < kOffThreads; o <<= 1) {  // inclusive scan (Hillis-Steele)
      const uint32_t y = t >= o ? sh[t - o] : 0u;
      __syncthreads();
      sh[t] += y;
      __syncthreads();
    }
    uint32_t pos = base + sh[t] - v;
#pragma unroll
    for (uint32_t i = 0; i < per; ++i) {
      P.chain_hist[c * kChainBins + t * per + i] = pos;
      pos += h[i];
    }
    __syncthreads();
    if (t == 0) {
      const uint32_t end = base + sh[kOffThreads - 1], padded = (end + 31u) & ~31u;
      for (uint32_t x = end; x < padded; ++x) P.rec[x].tile = kNoChain;
      base = padded;
      if (c == 3) P.lane_w[0] = padded / 32;
      if (c == kChainClasses - 1) P.lane_w[1] = padded / 32;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kTileThreads) k_chain_scatter(Plan P) {
  __shared__ uint32_t shT[kTileRows][33], shK[kTileRows][33], shF[kTileRows][33];
  __shared__ uint64_t shLo[kTileRows][33], shCnt[kTileRows][33];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t nt = tile_count(P), nst = (P.n + 31) / 32;
  for (size_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const TileIdx ti = tile_load_idx(P, tile);
    uint32_t T = 0, key = 0, f = 0;
    uint64_t lo = 0, cnt = 0;
    if (ti.ok) {
      const uint32_t s = ti.slot * P.rows_pp + ti.j;
      T = P.seg_tiles[s];
      if (T) {
        key = P.chain_key[s];
        f = P.seg_first[s];
        lo = P.seg_lo[s];
        cnt = P.seg_cnt[s];
      }
    }
    {
      const uint32_t r = threadIdx.x % kTileRows, c = threadIdx.x / kTileRows;
      shT[r][c] = T;
      shK[r][c] = key;
      shF[r][c] = f;
      shLo[r][c] = lo;
      shCnt[r][c] = cnt;
    }
    __syncthreads();
    T = shT[w][lane];
    key = shK[w][lane];
    f = shF[w][lane];
    lo = shLo[w][lane];
    cnt = shCnt[w][lane];
    __syncthreads();
    const uint32_t slot = (uint32_t)(tile % nst) * 32 + lane;
    const uint32_t row = (uint32_t)(tile / nst) * kTileRows + w;
    const uint32_t peers = __match_any_sync(0xffffffffu, T == 1 ? key : 0xffff0000u | lane);
    const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
    uint32_t pos = 0;
    if (T == 1 && lane == leader) pos = atomicAdd(&P.chain_hist[key], (uint32_t)__popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, (int)leader);
    if (T == 1) {
      P.rec[pos + __popc(peers & ((1u << lane) - 1u))] = PieceRec{lo, (uint32_t)cnt, f, slot, row};
    } else if (T > 1) {
      const uint32_t at = atomicAdd(&P.chain_hist[key], T);
      for (uint32_t k = 0; k < T; ++k) {
        const uint64_t b0 = cnt * k / T, b1 = cnt * (k + 1) / T;
        P.rec[at + k] = PieceRec{lo + b0, (uint32_t)(b1 - b0), f + k, slot, row};
      }
    }
  }
}

// tiles a plan of ns segments may hold: with lane chains sum_s ceil(cnt_s / L)
// is at most the chains wanted per path plus the segments (L >= a path's
// terms / its chains wanted); warp tiles: max_tiles per segment
static size_t tiles_capacity(const ResidueConfig &cfg, size_t ns, uint32_t max_tiles, int sms,
                             uint64_t rounds) {
  if (!cfg.lane_chains()) return ns * max_tiles;
  return ns + (size_t)sms * (kLaneThreads31 + kLaneThreads64) * rounds;
}

// Chain lengths of a serving plan from upper bounds t[path] on its terms:
// t / (kLaneRoundsEpoch x the path's resident lanes), within [floor, lmax];
// the plan then holds at most segments + sum t / L tiles.
static void epoch_chain_lengths(const double *t, int sms, uint64_t lmax, uint64_t *L,
                                size_t *extra_tiles) {
  const uint64_t lanes[2] = {(uint64_t)sms * kLaneThreads31, (uint64_t)sms * kLaneThreads64};
  const uint64_t lmin[2] = {kLaneMin31, kLaneMin64};
  *extra_tiles = 0;
  for (int i = 0; i < 2; ++i) {
    const double want = t[i] / (double)(kLaneRoundsEpoch * lanes[i]);
    uint64_t l = want > (double)lmax ? lmax : (uint64_t)want + 1;
    L[i] = l < lmin[i] ? lmin[i] : l;
    *extra_tiles += (size_t)(t[i] / (double)L[i]) + 1;
  }
}

// the lane-chain fields of a plan whose other buffers are set; `get`
// allocates device memory
template <typename Get>
static wv_status lane_setup(Plan &P, size_t tiles_cap, uint32_t *scal, int sms, uint64_t rounds,
                            Get get) {
  P.lane = 1;
  WV_CHECK(get((void **)&P.rec, (tiles_cap + 32 * kChainClasses) * sizeof(PieceRec)));
  WV_CHECK(get((void **)&P.chain_key, tiles_cap * sizeof(uint32_t)));
  WV_CHECK(get((void **)&P.chain_hist, (size_t)kChainClasses * kChainBins * sizeof(uint32_t)));
  WV_CHECK(get((void **)&P.lane_sum, 2 * sizeof(uint64_t)));
  P.lane_w = scal + 8;
  P.lane_target[0] = (uint64_t)sms * kLaneThreads31 * rounds;
  P.lane_target[1] = (uint64_t)sms * kLaneThreads64 * rounds;
  P.lane_min[0] = kLaneMin31;
  P.lane_min[1] = kLaneMin64;
  return WV_OK;
}

// the planner's launch sequence after the prime contexts: segments, pieces
// per segment, the tile map and, with lane chains, the sorted tile list
static wv_status plan_launches(Plan &P, uint32_t *u32tmp, int sms, cudaStream_t s) {
  const size_t ns = (size_t)P.n * P.rows_pp;
  WV_LAUNCH("plan_segments", k_plan_segments, (unsigned)((ns + 255) / 256), 256, 0, s, P);
  if (P.lane) {
    WV_CUDA(cudaMemsetAsync(P.lane_sum, 0, 2 * sizeof(uint64_t), s));
    WV_LAUNCH("lane_sum", k_lane_sum, (unsigned)(sms * 8), 256, 0, s, P);
    WV_LAUNCH("lane_chains", k_lane_chains, (unsigned)((ns + 255) / 256), 256, 0, s, P);
  }
  WV_CHECK(scan_exclusive_u32(P.seg_tiles, P.seg_first, ns, P.total_tiles, u32tmp, s));
  // the tile -> segment map serves warp tiles; lane chains read piece records
  if (!P.lane)
    WV_LAUNCH("plan_tilemap", k_plan_tilemap, (unsigned)((ns + 255) / 256), 256, 0, s, P);
  WV_LAUNCH("plan_split", k_plan_split, 1, 1, 0, s, P);
  if (P.lane) {
    // one tile of kTileRows rows by 32 primes per block (grid-stride beyond
    // 2^20 blocks): many warps in flight hide the atomics' latency
    const size_t gsz = (size_t)((P.rows_pp + kTileRows - 1) / kTileRows) * ((P.n + 31) / 32);
    const unsigned gs = (unsigned)(gsz < (1u << 20) ? (gsz ? gsz : 1) : (1u << 20));
    WV_CUDA(cudaMemsetAsync(P.chain_hist, 0, (size_t)kChainClasses * kChainBins * 4, s));
    WV_LAUNCH("chain_hist", k_chain_hist, gs, kTileThreads, 0, s, P);
    WV_LAUNCH("chain_offsets", k_chain_offsets, 1, kOffThreads, 0, s, P);
    WV_LAUNCH("chain_scatter", k_chain_scatter, gs, kTileThreads, 0, s, P);
  }
  return WV_OK;
}

// ------------------------------------------------------------------ finalize
__device__ __forceinline__ int64_t smod64(int64_t c, int64_t p) {
  int64_t r = c % p;
  return r < 0 ? r + p : r;
}

// B_{p-3}, E_{p-3} mod p for p = 5, 7 (where some LHS constants vanish):
// B_2 = 1/6 = 1 mod 5, E_2 = 1;  B_4 = -1/30 = 3 mod 7, E_4 = 5.
__device__ __forceinline__ uint64_t special_value(uint64_t p, bool isB) {
  if (p == 5) return 1;
  if (p == 7) return isB ? 3 : 5;
  return WV_RESIDUE_INVALID;
}

// One block per (prime, kind): its threads compute the powers d^-e of the
// congruence's bases and fold the sums' partials into fractions side by side,
// and the block merges the fractions (a prime's thousands of sums would make
// one warp's serial chain the launch's critical path).
constexpr int kFinThreads = 256;
__global__ void __launch_bounds__(kFinThreads) k_finalize(Plan P) {
  const int lane = threadIdx.x & 31;
  const uint32_t item = blockIdx.x;  // (slot, kind), uniform over the block
  const uint32_t nk = (P.rows_b ? 1u : 0u) + (P.rows_e ? 1u : 0u);
  if (item >= P.n * nk) return;
  const uint32_t slot = item / nk, kk = item - slot * nk;
  const bool isB = (P.rows_b != 0) && kk == 0;
  uint64_t *out = isB ? P.out_b : P.out_e;
  if (!out) return;
  const PrimeCtx ctx = P.ctx[slot];
  const uint32_t ge = isB ? P.gen_e_b : P.gen_e_e;  // general index: exponent e, else 0
  if (ctx.flags & 2u) {
    if (threadIdx.x == 0) out[ctx.orig] = ge ? WV_RESIDUE_INVALID : special_value(ctx.p, isB);
    return;
  }
  const Mont M(ctx);
  const int64_t p = (int64_t)ctx.p;
  if (ge && ctx.p < (uint64_t)ge + 3) {  // the general forms need 2 <= 2k <= p - 3
    if (threadIdx.x == 0) out[ctx.orig] = WV_RESIDUE_INVALID;
    return;
  }
  const uint32_t nrows = isB ? P.rows_b : P.rows_e;
  const uint32_t r0 = isB ? 0u : P.rows_b;
  const uint32_t seg0 = slot * P.rows_pp + r0;
  // d^-ex for the congruence's distinct bases d, once per prime and kind
  __shared__ int64_t dpow[kMaxDist];
  {
    const uint32_t d0 = isB ? P.db0 : P.de0, nd = isB ? P.dbn : P.den;
    const uint64_t ex = isB ? P.ex_b : P.ex_e;
    for (uint32_t i = threadIdx.x; i < nd; i += kFinThreads)
      dpow[i] = M.pow(M.to_mont((int64_t)(P.cg_dist[d0 + i] % ctx.p)), ctx.p - 1 - ex);
    __syncthreads();
  }
  const uint32_t reg0 = isB ? P.rb0 : P.re0;
  int64_t N = 0, D = M.one;  // running fraction N / D = sum coef_j c1_j / c0_j
  for (uint32_t j = threadIdx.x; j < nrows; j += kFinThreads) {
    const uint32_t s = seg0 + j;
    int64_t C0 = M.one, C1 = 0;
    const uint32_t f = P.seg_first[s], T = P.seg_tiles[s];
    for (uint32_t g = f; g < f + T; ++g) {
      const ulonglong2 v = P.partials[g];
      M.combine(C0, C1, (int64_t)v.x, (int64_t)v.y);
    }
    // coefficient sum_k c_k d_k^-ex, in Montgomery form
    const uint32_t *w = P.cg_rows + 6 * (size_t)(reg0 + j);
    int64_t aM = 0;
    for (uint32_t t = w[4]; t < w[4] + w[5]; ++t) {
      // most coefficients are +-1 (every one of the generated Bernoulli
      // congruences'), and all are far below p except at tiny p
      const int64_t c = P.cg_tc[t], dp = dpow[P.cg_td[t]];
      if (c == 1) {
        aM = M.add(aM, dp);
      } else if (c == -1) {
        aM = M.sub(aM, dp);
      } else {
        const int64_t cm = (c >= 0 && c < p) ? c : (c < 0 && -c < p) ? c + p : smod64(c, p);
        aM = M.add(aM, M.mul(M.to_mont(cm), dp));
      }
    }
    const int64_t X = M.mul(aM, C1);  // coef * C1 at C1's scale
    N = M.add(M.mul(N, C0), M.mul(X, D));
    D = M.mul(D, C0);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const int64_t N2 = __shfl_xor_sync(0xffffffffu, N, o);
    const int64_t D2 = __shfl_xor_sync(0xffffffffu, D, o);
    N = M.add(M.mul(N, D2), M.mul(N2, D));
    D = M.mul(D, D2);
  }
  __shared__ int64_t sN[kFinThreads / 32], sD[kFinThreads / 32];
  if (lane == 0) {
    sN[threadIdx.x >> 5] = N;
    sD[threadIdx.x >> 5] = D;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kFinThreads / 32; ++w) {
      N = M.add(M.mul(N, sD[w]), M.mul(sN[w], D));
      D = M.mul(D, sD[w]);
    }
    int64_t L;  // the constant on the left, plain
    if (ge && isB) {
      // C_k(a,b,c) = (a^e + b^e - c^e - 1) / (4k) with 4k = 2(p - e) = -2e (mod p):
      // the numerator stays in L, the denominator moves into N
      int64_t num = M.sub(0, M.one);
      for (int i = 0; i < 3; ++i) {
        const int64_t pw = M.pow(M.to_mont((int64_t)P.glhs[i]), ge);
        num = (i < 2) ? M.add(num, pw) : M.sub(num, pw);
      }
      L = M.from_mont(num);
      N = M.mul(N, M.to_mont(smod64(-2 * (int64_t)ge, p)));
    } else if (ge) {
      // (-1)^k 4^{2k-1} with 2k = e
      const int64_t f = M.from_mont(M.pow(M.to_mont(4), ge - 1));
      L = ((ge / 2) & 1) ? (f ? p - f : 0) : f;
    } else {
      L = smod64(isB ? P.lhs_b : P.lhs_e, p);
    }
    if (L == 0 || D == 0) {
      out[ctx.orig] = WV_RESIDUE_INVALID;
      return;
    }
    // residue = (N/D) R^-1 / L = N / (D L R)
    const int64_t DLR = M.mul(D, M.to_mont(M.to_mont(L)));  // D * L R^2 * R^-1
    const int64_t inv = M.pow(M.to_mont(DLR), (uint64_t)(p - 2));  // (DLR)^-1 R
    out[ctx.orig] = (uint64_t)M.mul(N, inv);                 // N (DLR)^-1
  }
}

// ------------------------------------------------------------------ host
// Tile shape of a plan of n primes with `rows` sums each.  With the library
// default (tiles_auto) a plan of few primes gets more and shorter tiles, so
// that one launch still holds about kTargetTiles tiles (several per resident
// warp) and its tail stays short: max_tiles grows up to 64 and tile_terms
// shrinks in proportion (not below 2^15).  Many primes keep the configured
// shape.  The partials buffer is bounded by max(n rows max_tiles, ~kTargetTiles).
constexpr size_t kTargetTiles = 98304;
static void tile_shape(const ResidueConfig &cfg, size_t n, size_t rows, uint32_t *tile_terms,
                       uint32_t *max_tiles) {
  uint32_t tt = (uint32_t)(cfg.tile_terms > 0 ? cfg.tile_terms : (1 << 20));
  uint32_t mt = (uint32_t)(cfg.max_tiles > 0 ? cfg.max_tiles : 8);
  if (cfg.tiles_auto && n > 0 && rows > 0) {
    const size_t want = (kTargetTiles + n * rows - 1) / (n * rows);
    if (want > mt) {
      const uint32_t m2 = (uint32_t)(want < 64 ? want : 64);
      const uint64_t t2 = (uint64_t)tt * mt / m2;
      tt = (uint32_t)(t2 < (1u << 15) ? (1u << 15) : t2);
      mt = m2;
    }
  }
  *tile_terms = tt;
  *max_tiles = mt;
}

AccKernel acc_kernel_m31(int ar, int ilp) {
  if (ar == 23) return k_accumulate<false, 1, 23>;  // the paper's arithmetic (ablation)
  if (ar == 24) return k_accumulate<false, 1, 24>;  // general index (wv_residues_general)
#define WV_PICK(I)                                                            \
  (ar == 1 ? k_accumulate<false, I, 1> : ar == 2 ? k_accumulate<false, I, 2> \
   : ar == 4 ? k_accumulate<false, I, 4> : k_accumulate<false, I, 9>)
  if (ar >= 25) return acc_kernel_m31x(ar, ilp);
  if (ilp == 1) return WV_PICK(1);
  if (ilp == 2) return WV_PICK(2);
#undef WV_PICK
  return k_accumulate<false, 4, 9>;
}

template <bool WIDE>
static wv_status launch_accumulate(const Plan &P, const ResidueConfig &cfg, int sms, cudaStream_t s) {
  const char *name = WIDE ? "accumulate_m64" : "accumulate_m31";
  AccKernel kern = nullptr;
  if (P.lane) {
    kern = WIDE ? acc_kernel_lane64(cfg.arith) : acc_kernel_lane31(cfg.arith, cfg.ilp);
  } else if (WIDE) {
    // arith 25..28 vary the 32-bit path only; the 64-bit path runs its default
    // the single-term forms (1, 2, 4) run the single-term 64-bit kernel, 12..18,
    // 21, 23..24 and 32..36 their own 64-bit forms, everything else the grouped
    // default
    kern = ((cfg.arith > 9 && cfg.arith <= 24) || cfg.arith >= 32)
               ? acc_kernel_m64x(cfg.arith, cfg.ilp64)
               : acc_kernel_m64(cfg.arith >= 9 ? 9 : 1, cfg.ilp64);
  } else {
    kern = acc_kernel_m31(cfg.arith >= 23 ? cfg.arith : cfg.arith > 9 ? 9 : cfg.arith, cfg.ilp);
  }
  int occ = cfg.blocks_per_sm;
  if (occ <= 0) {
    WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.block, 0));
    if (occ < 1) occ = 1;
  }
  WV_LAUNCH(name, kern, (unsigned)(sms * occ), cfg.block, 0, s, P);
  return WV_OK;
}

static void fill_rows(Plan &P, const ResidueConfig &cfg, const DeviceState *dev);

wv_status residues_device(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                          uint64_t *d_out_e, const ResidueConfig &cfg, cudaStream_t s) {
  if (n == 0) return WV_OK;
  if (!d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));
  Plan P;
  memset(&P, 0, sizeof P);
  P.check = cfg.check_primes ? 1u : 0u;
  const bool do_b = (cfg.gen_e_b ? true : cfg.cong_b >= 0) && d_out_b;
  const bool do_e = (cfg.gen_e_e ? true : cfg.cong_e >= 0) && d_out_e;
  if (!do_b && !do_e) return WV_OK;
  ResidueConfig c2 = cfg;
  if (!do_b) c2.cong_b = -2, c2.gen_e_b = 0;
  if (!do_e) c2.cong_e = -2, c2.gen_e_e = 0;
  fill_rows(P, c2, dev);

  const size_t cap = cfg.chunk > 0 ? (size_t)cfg.chunk : kChunkPrimes;
  const uint32_t chunk = (uint32_t)(n < cap ? n : cap);
  tile_shape(cfg, chunk, P.rows_pp, &P.tile_terms, &P.max_tiles);
  const size_t nseg = (size_t)chunk * P.rows_pp;
  Scratch sc(s);
  uint32_t *u32tmp = nullptr, *scal = nullptr;
  WV_CHECK(sc.get(&P.ctx, chunk));
  WV_CHECK(sc.get(&P.flag, chunk));
  WV_CHECK(sc.get(&P.pos, chunk));
  WV_CHECK(sc.get(&P.seg_lo, nseg));
  WV_CHECK(sc.get(&P.seg_cnt, nseg));
  WV_CHECK(sc.get(&P.seg_tiles, nseg));
  WV_CHECK(sc.get(&P.seg_first, nseg));
  const size_t tiles_cap = tiles_capacity(cfg, nseg, P.max_tiles, dev->sms, kLaneRounds);
  WV_CHECK(sc.get(&P.partials, tiles_cap));
  WV_CHECK(sc.get(&P.tile_seg, tiles_cap));
  WV_CHECK(sc.get(&u32tmp, scan_tmp_elems(nseg)));
  WV_CHECK(sc.get(&scal, 256));
  P.bk = scal + 64;
  P.n31 = scal + 0;
  P.total_tiles = scal + 1;
  P.split_tile = scal + 2;
  P.counters = scal + 4;
  if (cfg.lane_chains())
    WV_CHECK(lane_setup(P, tiles_cap, scal, dev->sms, kLaneRounds, [&](void **p, size_t bytes) {
      return sc.get((unsigned char **)p, bytes);
    }));

  for (size_t base = 0; base < n; base += chunk) {
    P.n = (uint32_t)((n - base) < chunk ? (n - base) : chunk);
    P.primes = d_primes + base;
    P.out_b = do_b ? d_out_b + base : nullptr;
    P.out_e = do_e ? d_out_e + base : nullptr;
    const unsigned gp = (P.n + 255) / 256;
    WV_CUDA(cudaMemsetAsync(P.bk, 0, 192 * sizeof(uint32_t), s));
    WV_LAUNCH("plan_prime", k_plan_prime, gp, 256, 0, s, P);
    WV_LAUNCH("plan_buckets", k_plan_buckets, 1, 32, 0, s, P);
    WV_LAUNCH("plan_scatter", k_plan_scatter, gp, 256, 0, s, P);
    WV_CHECK(plan_launches(P, u32tmp, dev->sms, s));
    WV_CHECK(launch_accumulate<false>(P, cfg, dev->sms, s));
    WV_CHECK(launch_accumulate<true>(P, cfg, dev->sms, s));
    const uint32_t nk = (do_b ? 1 : 0) + (do_e ? 1 : 0);
    const size_t items = (size_t)P.n * nk;  // one block per (prime, kind)
    WV_LAUNCH("finalize", k_finalize, (unsigned)items, kFinThreads, 0, s, P);
  }
  return WV_OK;
}

// ------------------------------------------------------------------ phases
// The launch sequence of residues_device split into its phases, for callers
// that interleave the accumulation of several prime lists (the serving loop):
// plan_build -> plan_totals -> epoch_launch (any number of times, over any
// tile ranges) -> plan_finalize -> plan_free.

static void fill_rows(Plan &P, const ResidueConfig &cfg, const DeviceState *dev) {
  P.uform_min[0] = cfg.uform_min31;
  P.uform_min[1] = cfg.uform_min64;
  P.cg_rows = dev->cg_rows;
  P.cg_tc = dev->cg_tc;
  P.cg_td = dev->cg_td;
  P.cg_dist = dev->cg_dist;
  uint32_t r = 0;
  auto use = [&](int id, bool isB) {
    const CongView &v = cong_view(id);
    if (isB) {
      P.rows_b = (uint32_t)v.nrows;
      P.rb0 = v.row0;
      P.db0 = v.dist0;
      P.dbn = v.ndist;
      P.lhs_b = v.lhs;
    } else {
      P.rows_e = (uint32_t)v.nrows;
      P.re0 = v.row0;
      P.de0 = v.dist0;
      P.den = v.ndist;
      P.lhs_e = v.lhs;
    }
    r += (uint32_t)v.nrows;
  };
  if (cfg.gen_e_b) {
    use(cong_general_id(0), true);
    P.gen_e_b = P.ex_b = cfg.gen_e_b;
    for (int i = 0; i < 3; ++i) P.glhs[i] = kWvGeneral[0].lhs[i];
  } else if (cfg.cong_b >= 0) {
    use(cfg.cong_b, true);
    P.ex_b = 3;  // t = p - 4: d^t = d^-3
  }
  if (cfg.gen_e_e) {
    use(cong_general_id(1), false);
    P.gen_e_e = P.ex_e = cfg.gen_e_e;
  } else if (cfg.cong_e >= 0) {
    use(cfg.cong_e, false);
    P.ex_e = 2;  // t = p - 3: d^t = d^-2
  }
  P.rows_pp = r;
}

static size_t rows_of(const ResidueConfig &cfg) {
  size_t r = 0;
  if (cfg.gen_e_b) r += cong_view(cong_general_id(0)).nrows;
  else if (cfg.cong_b >= 0) r += cong_view(cfg.cong_b).nrows;
  if (cfg.gen_e_e) r += cong_view(cong_general_id(1)).nrows;
  else if (cfg.cong_e >= 0) r += cong_view(cfg.cong_e).nrows;
  return r;
}

size_t plan_bytes(uint32_t n, const ResidueConfig &cfg, const double *terms) {
  const size_t ns = (size_t)n * rows_of(cfg);
  uint32_t tt = 0, mt = 0;
  tile_shape(cfg, n, rows_of(cfg), &tt, &mt);
  DeviceState *dev = nullptr;
  const int sms = device_state(&dev) == WV_OK ? dev->sms : 160;
  size_t tc = tiles_capacity(cfg, ns, mt, sms, kLaneRoundsEpoch);
  if (cfg.lane_chains() && terms) {
    uint64_t L[2];
    size_t extra = 0;
    epoch_chain_lengths(terms, sms, cfg.epoch_piece_max, L, &extra);
    tc = ns + extra;
  }
  size_t b = n * (sizeof(PrimeCtx) + 8) + ns * (8 + 8 + 4 + 4) + tc * (sizeof(ulonglong2) + 4) +
             scan_tmp_elems(ns) * 4 + 1024 + 16 * 256;
  if (cfg.lane_chains())  // sorted tile list, keys, bins, terms per path
    b += tc * 8 + 32 * kChainClasses * 4 + (size_t)kChainClasses * kChainBins * 4 + 16 + 4 * 256;
  return b;
}

size_t plan_struct_bytes() { return sizeof(Plan); }

wv_status plan_build(const uint64_t *d_primes, uint32_t n, const ResidueConfig &cfg, PlanState *ps,
                     cudaStream_t s, const double *terms) {
  if (n == 0 || n > 65536) return set_error(WV_EINVAL, "plan_build: n=%u not in [1, 65536]", n);
  DeviceState *dev = nullptr;
  WV_CHECK(device_state(&dev));
  ps->host = new Plan();
  Plan &P = *ps->host;
  memset(&P, 0, sizeof P);
  P.check = cfg.check_primes ? 1u : 0u;
  fill_rows(P, cfg, dev);
  tile_shape(cfg, n, P.rows_pp, &P.tile_terms, &P.max_tiles);
  const size_t ns = (size_t)n * P.rows_pp;
  auto get = [&](void **p, size_t bytes) -> wv_status {
    WV_CHECK(scratch_alloc(p, bytes + 256, s));
    ps->blocks[ps->nblocks++] = *p;
    ps->bytes += bytes + 256;
    return WV_OK;
  };
  uint32_t *u32tmp = nullptr, *scal = nullptr;
  WV_CHECK(get((void **)&P.ctx, n * sizeof(PrimeCtx)));
  WV_CHECK(get((void **)&P.flag, n * 4));
  WV_CHECK(get((void **)&P.seg_lo, ns * 8));
  WV_CHECK(get((void **)&P.seg_cnt, ns * 8));
  WV_CHECK(get((void **)&P.seg_tiles, ns * 4));
  WV_CHECK(get((void **)&P.seg_first, ns * 4));
  size_t tiles_cap = tiles_capacity(cfg, ns, P.max_tiles, dev->sms, kLaneRoundsEpoch);
  if (cfg.lane_chains() && terms) {
    size_t extra = 0;
    epoch_chain_lengths(terms, dev->sms, cfg.epoch_piece_max, P.lane_fix, &extra);
    tiles_cap = ns + extra;
  }
  WV_CHECK(get((void **)&P.partials, tiles_cap * sizeof(ulonglong2)));
  WV_CHECK(get((void **)&P.tile_seg, tiles_cap * sizeof(uint32_t)));
  WV_CHECK(get((void **)&u32tmp, scan_tmp_elems(ns) * 4));
  WV_CHECK(get((void **)&scal, 1024));
  P.pos = nullptr;
  P.bk = scal + 64;
  P.n31 = scal + 0;
  P.total_tiles = scal + 1;
  P.split_tile = scal + 2;
  P.counters = scal + 4;
  if (cfg.lane_chains()) WV_CHECK(lane_setup(P, tiles_cap, scal, dev->sms, kLaneRoundsEpoch, get));
  P.n = n;
  P.primes = d_primes;
  ps->n = n;
  const unsigned gp = (n + 255) / 256;
  WV_CUDA(cudaMemsetAsync(P.bk, 0, 192 * sizeof(uint32_t), s));
  WV_LAUNCH("plan_prime", k_plan_prime, gp, 256, 0, s, P);
  WV_LAUNCH("plan_buckets", k_plan_buckets, 1, 32, 0, s, P);
  WV_LAUNCH("plan_scatter", k_plan_scatter, gp, 256, 0, s, P);
  return plan_launches(P, u32tmp, dev->sms, s);
}

// A plan's work units and the first unit of the 64-bit kernel: tiles, or
// with lane chains warps of the sorted tile list (lane_w at scal + 8).
wv_status plan_totals(PlanState *ps, cudaStream_t s) {
  uint32_t v[10] = {};
  uint64_t t[2] = {0, 0};
  WV_CUDA(cudaMemcpyAsync(v, ps->host->n31, 10 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (ps->host->lane)
    WV_CUDA(cudaMemcpyAsync(t, ps->host->lane_sum, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  WV_CUDA(cudaStreamSynchronize(s));
  ps->total = ps->host->lane ? v[9] : v[1];
  ps->split = ps->host->lane ? v[8] : v[2];
  if (ps->host->lane) ps->terms[0] = (double)t[0], ps->terms[1] = (double)t[1];
  return WV_OK;
}

wv_status plan_upload(const PlanState *ps, Plan *d_plan, cudaStream_t s) {
  WV_CUDA(cudaMemcpyAsync(d_plan, ps->host, sizeof(Plan), cudaMemcpyHostToDevice, s));
  return WV_OK;
}

wv_status epoch_launch(bool wide, const EpochItem *d_items, uint32_t n_items, uint32_t total,
                       const Plan *d_plans, uint32_t *d_counter, const ResidueConfig &cfg, int sms,
                       int reserve_blocks, cudaStream_t s) {
  if (total == 0) return WV_OK;
  EpochKernel kern = epoch_kernel(wide, wide ? cfg.ilp64 : cfg.ilp, cfg.lane_chains());
  int occ = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.block, 0));
  if (occ < 1) occ = 1;
  WV_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s));
  // reserve_blocks is counted in 256-thread blocks
  int grid = sms * occ - reserve_blocks * (kAccThreads / cfg.block);
  if (grid < 1) grid = 1;
  WV_LAUNCH(wide ? "epoch_m64" : "epoch_m31", kern, (unsigned)grid, cfg.block, 0, s,
            d_items, n_items, total, d_plans, d_counter);
  return WV_OK;
}

wv_status epoch_launch_mixed(const EpochItem *d_items, uint32_t n_items, uint32_t total,
                             const Plan *d_plans, uint32_t *d_counter, const ResidueConfig &cfg,
                             int sms, int reserve_blocks, cudaStream_t s) {
  if (total == 0) return WV_OK;
  EpochKernel kern = epoch_mixed_kernel(cfg.ilp, cfg.ilp64, cfg.lane_chains());
  int occ = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.block, 0));
  if (occ < 1) occ = 1;
  WV_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s));
  // reserve_blocks is counted in warps' worth of 256-thread blocks
  int grid = sms * occ - reserve_blocks * (kAccThreads / cfg.block);
  if (grid < 1) grid = 1;
  WV_LAUNCH("epoch", kern, (unsigned)grid, cfg.block, 0, s, d_items, n_items, total, d_plans,
            d_counter);
  return WV_OK;
}

wv_status epoch_launch_tiles(const EpochItem *d_items, uint32_t n_items, uint32_t total,
                             const Plan *d_plans, const ResidueConfig &cfg, cudaStream_t s) {
  if (total == 0) return WV_OK;
  const uint32_t wpb = (uint32_t)(cfg.block / 32);
  WV_LAUNCH("epoch", epoch_tiles_kernel(cfg.ilp, cfg.lane_chains()), (total + wpb - 1) / wpb, cfg.block, 0, s, d_items,
            n_items, total, d_plans);
  return WV_OK;
}

wv_status plan_finalize(PlanState *ps, uint64_t *d_out_b, uint64_t *d_out_e, cudaStream_t s) {
  Plan P = *ps->host;
  P.out_b = P.rows_b ? d_out_b : nullptr;
  P.out_e = P.rows_e ? d_out_e : nullptr;
  const uint32_t nk = (P.rows_b ? 1u : 0u) + (P.rows_e ? 1u : 0u);
  const size_t items = (size_t)P.n * nk;
  WV_LAUNCH("finalize", k_finalize, (unsigned)items, kFinThreads, 0, s, P);
  return WV_OK;
}

void plan_free(PlanState *ps, cudaStream_t s) {
  for (int i = ps->nblocks - 1; i >= 0; --i) scratch_free(ps->blocks[i], s);
  ps->nblocks = 0;
  ps->bytes = 0;
  delete ps->host;
  ps->host = nullptr;
}

// ------------------------------------------------------------------ no-alloc
// Residues without any allocation: every scratch buffer of the launch sequence
// above is carved from one file-scope device array of fixed size instead of
// the library's stream-ordered pool.  Sized for kNoAllocMaxPrimes primes per
// call with the default congruences and launch shape (max_tiles 8).
constexpr uint32_t kNoAllocMaxPrimes = 1024;
constexpr uint32_t kNoAllocTiles = 8;

__host__ __device__ constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaSegs = (size_t)kNoAllocMaxPrimes * kMaxRowsPP;
constexpr size_t kNaScanTmp = kNaSegs / 4096 + 2;  // scan_tmp_elems bound for kNaSegs
constexpr size_t kNaBytes =
    na_align(kNoAllocMaxPrimes * sizeof(PrimeCtx)) + 2 * na_align(kNoAllocMaxPrimes * 4) +
    2 * na_align(kNaSegs * 8) + 2 * na_align(kNaSegs * 4) +
    na_align(kNaSegs * kNoAllocTiles * sizeof(ulonglong2)) +
    na_align(kNaSegs * kNoAllocTiles * sizeof(uint32_t)) + na_align(kNaScanTmp * 4) + 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// BB30 + EE33 in registry form (63 rows, one term each, base 1), written
// once per device at the first call
static __device__ uint32_t g_na_rows[kMaxRowsPP * 6];
static __device__ int64_t g_na_tc[kMaxRowsPP];
static __device__ uint16_t g_na_td[kMaxRowsPP];
static __device__ uint64_t g_na_dist[2];
static std::mutex g_na_mu;
static void *g_na_addr[64];  // device address of g_noalloc_scratch, per device
static void *g_na_cg[64][4];  // device addresses of the four arrays above, per device

wv_status residues_noalloc(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                           uint64_t *d_out_e, cudaStream_t s) {
  if (n == 0) return WV_OK;
  if (!d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  if (n > kNoAllocMaxPrimes)
    return set_error(WV_ERANGE, "wv_residues_pm3_noalloc takes at most %u primes per call (got %zu)",
                     kNoAllocMaxPrimes, n);
  const bool do_b = d_out_b != nullptr, do_e = d_out_e != nullptr;
  if (!do_b && !do_e) return WV_OK;
  int dev = 0;
  WV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(WV_EINVAL, "device index %d out of range", dev);
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
      // The array's name is only a host-side stand-in: its device address
      // must be looked up once per device, with that device current.
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
      // the congruence rows, copied into their static arrays (no allocation).
      // The arrays hold at most kMaxRowsPP rows of one term each with base
      // d = 1; a congruence outside that shape is refused, not truncated.
      uint32_t nrows_all = 0;
      for (int id : {kWvDefaultB, kWvDefaultE}) {
        const CongView &v = cong_view(id);
        nrows_all += (uint32_t)v.nrows;
        bool ok = v.ndist == 1 && cong_dist()[v.dist0] == 1;
        for (int j = 0; ok && j < v.nrows; ++j) ok = cong_row(v.row0 + j)[5] == 1;
        if (!ok)
          return set_error(WV_EINVAL, "internal: congruence %s does not fit the no-alloc tables",
                           v.name);
      }
      if (nrows_all > (uint32_t)kMaxRowsPP)
        return set_error(WV_EINVAL, "internal: %u congruence rows exceed the no-alloc tables (%d)",
                         nrows_all, kMaxRowsPP);
      uint32_t rows[kMaxRowsPP * 6];
      int64_t tc[kMaxRowsPP];
      uint16_t td[kMaxRowsPP];
      const uint64_t dist[2] = {1, 1};
      uint32_t r = 0;
      for (int id : {kWvDefaultB, kWvDefaultE}) {
        const CongView &v = cong_view(id);
        for (int j = 0; j < v.nrows; ++j, ++r) {
          const uint32_t *w = cong_row(v.row0 + j);
          rows[6 * r + 0] = w[0];
          rows[6 * r + 1] = w[1];
          rows[6 * r + 2] = w[2];
          rows[6 * r + 3] = w[3];
          rows[6 * r + 4] = r;
          rows[6 * r + 5] = 1;
          tc[r] = cong_tc()[w[4]];
          td[r] = 0;  // base d = 1, index 0 of each congruence's own list
        }
      }
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_na_rows, rows, sizeof rows);
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_na_tc, tc, sizeof tc);
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_na_td, td, sizeof td);
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_na_dist, dist, sizeof dist);
      // A copy from pageable host memory may return before it has reached the
      // device, and a caller's non-blocking stream is not ordered after it:
      // wait for the device once, here, so the first launch sees the rows.
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&g_na_cg[dev][0], g_na_rows);
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&g_na_cg[dev][1], g_na_tc);
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&g_na_cg[dev][2], g_na_td);
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&g_na_cg[dev][3], g_na_dist);
      if (e != cudaSuccess) return cuda_fail(e, "noalloc congruence tables");
      g_na_addr[dev] = ptr;
    }
    base = (unsigned char *)g_na_addr[dev];
  }
  int sms = 0;
  WV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  // BB30 + EE33 (63 rows), whatever the library default: the scratch array
  // is sized for them
  ResidueConfig cfg;
  cfg.cong_b = do_b ? kWvDefaultB : -2;
  cfg.cong_e = do_e ? kWvDefaultE : -2;
  Plan P;
  memset(&P, 0, sizeof P);
  uint32_t r = 0;
  if (do_b) {
    const CongView &v = cong_view(cfg.cong_b);
    P.rows_b = (uint32_t)v.nrows;
    P.lhs_b = v.lhs;
    P.ex_b = 3;
    r += P.rows_b;
  }
  if (do_e) {
    const CongView &v = cong_view(cfg.cong_e);
    P.rows_e = (uint32_t)v.nrows;
    P.lhs_e = v.lhs;
    P.ex_e = 2;
    r += P.rows_e;
  }
  P.rows_pp = r;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    P.cg_rows = (const uint32_t *)g_na_cg[dev][0];
    P.cg_tc = (const int64_t *)g_na_cg[dev][1];
    P.cg_td = (const uint16_t *)g_na_cg[dev][2];
    P.cg_dist = (const uint64_t *)g_na_cg[dev][3];
  }
  // rows: BB30 at 0 (base index 0), EE33 after it (base index 1)
  P.rb0 = 0;
  P.re0 = (uint32_t)cong_view(kWvDefaultB).nrows;
  P.db0 = 0;
  P.dbn = 1;
  P.de0 = 1;
  P.den = 1;
  P.tile_terms = (uint32_t)cfg.tile_terms;
  P.max_tiles = kNoAllocTiles;
  // carve the scratch array
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char *q = base + off;
    off += na_align(bytes);
    return q;
  };
  P.ctx = (PrimeCtx *)carve(kNoAllocMaxPrimes * sizeof(PrimeCtx));
  P.flag = (uint32_t *)carve(kNoAllocMaxPrimes * 4);
  P.pos = (uint32_t *)carve(kNoAllocMaxPrimes * 4);
  P.seg_lo = (uint64_t *)carve(kNaSegs * 8);
  P.seg_cnt = (uint64_t *)carve(kNaSegs * 8);
  P.seg_tiles = (uint32_t *)carve(kNaSegs * 4);
  P.seg_first = (uint32_t *)carve(kNaSegs * 4);
  P.partials = (ulonglong2 *)carve(kNaSegs * kNoAllocTiles * sizeof(ulonglong2));
  P.tile_seg = (uint32_t *)carve(kNaSegs * kNoAllocTiles * sizeof(uint32_t));
  uint32_t *u32tmp = (uint32_t *)carve(kNaScanTmp * 4);
  uint32_t *scal = (uint32_t *)carve(256 * sizeof(uint32_t));
  if (off > kNaBytes) return set_error(WV_EINVAL, "internal: no-alloc scratch layout overflow");
  P.bk = scal + 64;
  P.n31 = scal + 0;
  P.total_tiles = scal + 1;
  P.split_tile = scal + 2;
  P.counters = scal + 4;  // zeroed by k_plan_split before every accumulation
  P.n = (uint32_t)n;
  P.primes = d_primes;
  P.out_b = do_b ? d_out_b : nullptr;
  P.out_e = do_e ? d_out_e : nullptr;

  const unsigned gp = (P.n + 255) / 256;
  const size_t ns = (size_t)P.n * P.rows_pp;
  WV_CUDA(cudaMemsetAsync(P.bk, 0, 192 * sizeof(uint32_t), s));
  k_plan_prime<<<gp, 256, 0, s>>>(P);
  k_plan_buckets<<<1, 32, 0, s>>>(P);
  k_plan_scatter<<<gp, 256, 0, s>>>(P);
  k_plan_segments<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(P);
  WV_CHECK(scan_exclusive_u32_bare(P.seg_tiles, P.seg_first, ns, P.total_tiles, u32tmp, s));
  k_plan_tilemap<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(P);
  k_plan_split<<<1, 1, 0, s>>>(P);
  WV_CUDA(cudaGetLastError());
  AccKernel k31 = acc_kernel_m31(9, 2);
  AccKernel k64 = acc_kernel_m64(9, 1);
  int occ31 = 0, occ64 = 0;
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ31, k31, kAccThreads, 0));
  WV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k64, kAccThreads, 0));
  k31<<<(unsigned)(sms * (occ31 > 0 ? occ31 : 1)), kAccThreads, 0, s>>>(P);
  k64<<<(unsigned)(sms * (occ64 > 0 ? occ64 : 1)), kAccThreads, 0, s>>>(P);
  const size_t items = (size_t)P.n * ((do_b ? 1 : 0) + (do_e ? 1 : 0));
  k_finalize<<<(unsigned)items, kFinThreads, 0, s>>>(P);
  WV_CUDA(cudaGetLastError());
  return WV_OK;
}

}  // namespace wv

using namespace wv;

extern "C" {

wv_status wv_residues_ex(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                         uint64_t *d_out_e, const wv_options *opt, wv_stream stream) {
  clear_error();
  if (n > 0 && !d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  if (n > ((size_t)1 << 40)) return set_error(WV_EINVAL, "n too large");
  ResidueConfig cfg;
  WV_CHECK(resolve_config(opt, d_out_b != nullptr, d_out_e != nullptr, &cfg));
  return residues_device(d_primes, n, d_out_b, d_out_e, cfg, (cudaStream_t)stream);
}

wv_status wv_residues_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                          uint64_t *d_out_e, wv_stream stream) {
  return wv_residues_ex(d_primes, n, d_out_b, d_out_e, nullptr, stream);
}

wv_status wv_bernoulli_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out, wv_stream stream) {
  if (n > 0 && !d_out) {
    clear_error();
    return set_error(WV_EINVAL, "d_out is NULL");
  }
  return wv_residues_ex(d_primes, n, d_out, nullptr, nullptr, stream);
}

wv_status wv_residues_pm3_noalloc(const uint64_t *d_primes, size_t n, uint64_t *d_out_b,
                                  uint64_t *d_out_e, wv_stream stream) {
  clear_error();
  return residues_noalloc(d_primes, n, d_out_b, d_out_e, (cudaStream_t)stream);
}

wv_status wv_residues_general(const uint64_t *d_primes, size_t n, uint32_t e_b, uint32_t e_e,
                              uint64_t *d_out_b, uint64_t *d_out_e, wv_stream stream) {
  clear_error();
  if (e_b && (e_b < 3 || e_b > kWvGeneralMaxE || !(e_b & 1)))
    return set_error(WV_EINVAL, "e_b=%u must be odd, 3 <= e_b <= %u (or 0)", e_b, kWvGeneralMaxE);
  if (e_e && (e_e < 2 || e_e > kWvGeneralMaxE || (e_e & 1)))
    return set_error(WV_EINVAL, "e_e=%u must be even, 2 <= e_e <= %u (or 0)", e_e, kWvGeneralMaxE);
  if (n && !d_primes) return set_error(WV_EINVAL, "d_primes is NULL");
  ResidueConfig cfg;
  WV_CHECK(resolve_config(nullptr, true, true, &cfg));
  cfg.arith = 24;
  cfg.ilp = cfg.ilp64 = 1;
  cfg.gen_e_b = e_b;
  cfg.gen_e_e = e_e;
  return residues_device(d_primes, n, e_b ? d_out_b : nullptr, e_e ? d_out_e : nullptr, cfg,
                         (cudaStream_t)stream);
}

wv_status wv_euler_pm3(const uint64_t *d_primes, size_t n, uint64_t *d_out, wv_stream stream) {
  if (n > 0 && !d_out) {
    clear_error();
    return set_error(WV_EINVAL, "d_out is NULL");
  }
  return wv_residues_ex(d_primes, n, nullptr, d_out, nullptr, stream);
}

}  // extern "C"
