// wv_serve.cu -- step a9: a continuous-batching serving loop (see include/wv_serve.h).
//
// Two threads per server:
//   * the admitter takes pending queries in arrival order and, as active
//     slots, plan slots and the device memory budget allow, gives each its
//     prime list (a range query is sieved on the device), residue buffers
//     and one plan per <= 65536 primes, all resident; it works on its own
//     high-priority stream, beside the running epochs;
//   * the worker runs epochs: the active queries, ordered by remaining work
//     (smallest first), contribute ranges of their not-yet-run tiles until
//     the epoch's term budget is filled, and one persistent launch runs all
//     of them (both arithmetic paths); two epochs are kept in flight on two
//     streams.  When an epoch retires, every plan whose tiles have all run is
//     finalised, and a query whose plans are all finalised is copied to the
//     host, marked done and its device memory released.
// A query admitted while others run joins the next epoch, so its tiles share
// launches with long-running ones.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/wv_serve.h"
#include "wv_internal.h"
#include "wv_tables.h"

namespace wv {

constexpr uint32_t kPlanPrimes = 65536;  // primes per plan
constexpr uint32_t kMaxPlans = 2048;     // plan slots per server
constexpr double kWideWeight = 3.0;      // cost of a 64-bit-path term relative to a 32-bit one
constexpr double kMinEpochTerms = 5e9;   // shortest epoch
constexpr size_t kAdmitScan = 4096;      // pending queries looked at per admission decision
constexpr double kAdmitAge = 5.0;        // seconds pending after which a query goes first
// Persistent epoch grids leave this many 256-thread blocks' room so that
// admission work (sieve, planner: small kernels) runs beside a running epoch.
constexpr int kReserveBlocks = 4;
constexpr int kEpochBlock = 32;          // default threads per block of an epoch launch

struct SChunk {  // one plan of a query; its tile state is the worker's
  PlanState plan;
  uint32_t off = 0, n = 0;
  uint32_t slot = 0;       // index in the device plan array
  int64_t last_epoch = -1; // last epoch that ran tiles of this plan
  uint32_t hi31 = 0;       // 32-bit-path tiles [0, hi31) not yet run
  uint32_t hi64 = 0;       // 64-bit-path tiles [split, hi64) not yet run
  double tpt31 = 1, tpt64 = 1;  // estimated terms per tile
  bool finalized = false;
};

struct SQuery {
  uint64_t id = 0;
  int kind = 0;
  uint64_t lo = 0, hi = 0;
  int state = 0;  // 0 pending, 1 active, 2 done, 3 failed, 4 cancelled
  wv_status status = WV_OK;
  std::string err;
  double t_submit = 0, t_admit = 0, t_done = 0;
  uint64_t *d_primes = nullptr, *d_rb = nullptr, *d_re = nullptr;
  size_t n = 0, bytes = 0;
  std::vector<SChunk> chunks;
  std::vector<uint64_t> h_primes, h_rb, h_re;
  uint64_t n_hits = 0;
  double remaining = 0;
  bool counted = false;          // bound on n and bytes known (admission)
  uint64_t n_cap = 0;            // capacity of d_primes (the admission bound)
  wv_status count_status = WV_OK;
};

static void terms_host(const uint64_t *ps, size_t n, const ResidueConfig &cfg, double *t31,
                       double *t64) {
  double a = 0, b = 0;
  for (size_t i = 0; i < n; ++i) {
    const uint64_t p = ps[i];
    if (p < 11 || p >= WV_P_MAX || !(p & 1)) continue;
    uint64_t t = 0;
    for (int kind = 0; kind < 2; ++kind) {
      const int id = kind ? cfg.cong_e : cfg.cong_b;
      if (id < 0) continue;
      const CongView &c = cong_view(id);
      for (int j = 0; j < c.nrows; ++j) t += cong_row_terms(c.row0 + j, p);
    }
    if (p < (1ull << 31)) a += (double)t;  // the 32-bit kernel takes p < 2^31
    else b += (double)t;
  }
  *t31 = a;
  *t64 = b;
}

// Upper bound on the number of primes in [lo, hi), for admission before the
// range is sieved: pi(x + y) - pi(x) <= 2y / log y for y > 1 (the
// Brun-Titchmarsh inequality in the form of Montgomery and Vaughan), and at
// most the odd numbers of a short range.
static uint64_t prime_count_bound(uint64_t lo, uint64_t hi) {
  const uint64_t y = hi > lo ? hi - lo : 0;
  const uint64_t odd = y / 2 + 2;
  if (y < 64) return odd;
  const uint64_t bt = (uint64_t)(2.0 * (double)y / std::log((double)y)) + 2;
  return bt < odd ? bt : odd;
}

}  // namespace wv

using namespace wv;

struct wv_server_s {
  wv_server_config cfg{};
  int device = 0, sms = 0;
  cudaStream_t sa = nullptr;       // admission: sieve, planning (high priority)
  cudaStream_t st = nullptr;       // finalisation, result copies (high priority)
  cudaStream_t se[2] = {};         // epochs alternate between two streams
  cudaEvent_t ev[2] = {};          // epoch completion
  std::thread worker, admitter;
  std::mutex mu;                   // guards everything below that both threads touch
  std::condition_variable cv_work, cv_admit, cv_done;
  std::deque<SQuery *> pending;    // submitted, not yet admitted (admitter pops)
  std::vector<SQuery *> active;    // admitted; tile state owned by the worker
  std::unordered_map<uint64_t, SQuery *> queries;
  bool stop = false;
  uint64_t next_id = 1;
  size_t bytes_in_use = 0;         // device bytes reserved by admitted queries
  Plan *d_plans = nullptr;
  std::vector<uint32_t> free_slots;
  EpochItem *d_items = nullptr, *h_items = nullptr;  // two halves, one per epoch stream
  uint32_t *d_counter = nullptr;                     // 2 x 2 counters
  ResidueConfig rcfg;
  std::chrono::steady_clock::time_point t0;
  uint64_t epochs = 0, tiles = 0;
  uint32_t peak_active = 0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Free a query's device memory (stream-ordered on s) and return its plan slots.
void release_device(wv_server_s *S, SQuery *q, cudaStream_t s) {
  std::vector<uint32_t> slots;
  for (auto &c : q->chunks) {
    if (c.plan.host) plan_free(&c.plan, s);
    slots.push_back(c.slot);
  }
  q->chunks.clear();
  scratch_free(q->d_primes, s);
  scratch_free(q->d_rb, s);
  scratch_free(q->d_re, s);
  q->d_primes = q->d_rb = q->d_re = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  for (uint32_t v : slots) S->free_slots.push_back(v);
}

// The configuration of a query: the server's, with the congruences for its
// primes (all below q->hi for a range, q->lo itself for a single prime).
ResidueConfig query_cfg(const wv_server_s *S, const SQuery *q) {
  ResidueConfig qc = S->rcfg;
  int cb = qc.cong_b, ce = qc.cong_e;
  cong_for_range(q->kind == 0 ? q->hi : q->lo + 1, &cb, &ce);
  qc.cong_b = cb;
  qc.cong_e = ce;
  return qc;
}

// Upper bounds on the terms of the n primes ps per kernel, in O(n): with
// W = the summed widths y - x of the congruences' rows, a prime holds at
// most W p + rows terms.
static void congruence_width(const ResidueConfig &cfg, double *w, double *rows);
static void terms_linear(const uint64_t *ps, size_t n, const ResidueConfig &cfg, double t[2]) {
  double w = 0, rows = 0, s31 = 0, s64 = 0, n31 = 0, n64 = 0;
  congruence_width(cfg, &w, &rows);
  for (size_t i = 0; i < n; ++i) {
    const uint64_t p = ps[i];
    if (p < (1ull << 31)) s31 += (double)p, n31 += 1;
    else s64 += (double)p, n64 += 1;
  }
  t[0] = w * s31 + rows * n31;
  t[1] = w * s64 + rows * n64;
}

// Upper bounds on the terms of m primes below pmax, per kernel (32-bit for
// p < 2^31, 64-bit above): a row (x, y) holds at most (y - x) p + 1 terms.
static void congruence_width(const ResidueConfig &cfg, double *w, double *rows) {
  *w = 0;
  *rows = 0;
  for (int kind = 0; kind < 2; ++kind) {
    const int id = kind ? cfg.cong_e : cfg.cong_b;
    if (id < 0) continue;
    const CongView &c = cong_view(id);
    for (int j = 0; j < c.nrows; ++j) {
      const uint32_t *r = cong_row(c.row0 + j);
      *w += (double)r[2] / r[3] - (double)r[0] / r[1];
    }
    *rows += c.nrows;
  }
}

static void terms_bound(const ResidueConfig &cfg, uint64_t m, uint64_t pmax, double t[2]) {
  double w = 0, rows = 0;
  congruence_width(cfg, &w, &rows);
  const double lo31 = std::min<double>((double)pmax, 2147483648.0);
  t[0] = (double)m * (w * lo31 + rows);
  t[1] = pmax > (1ull << 31) ? (double)m * (w * (double)pmax + rows) : 0.0;
}

// Device bytes a query of n primes holds while active.
size_t query_bytes(const wv_server_s *S, const SQuery *q, uint64_t n) {
  const ResidueConfig qc = query_cfg(S, q);
  const uint64_t pmax = q->kind == 0 ? q->hi : q->lo + 1;
  size_t need = n * 24;
  for (uint64_t off = 0; off < n; off += kPlanPrimes) {
    const uint32_t m = (uint32_t)std::min<uint64_t>(kPlanPrimes, n - off);
    double t[2];
    terms_bound(qc, m, pmax, t);
    need += plan_bytes(m, qc, t);
  }
  return need;
}

// Build an admitted query's device state on the admission stream: its
// primes (a range is sieved into a buffer sized by the bound used at
// admission), residue buffers, and one plan per kPlanPrimes primes in the
// reserved slots.  Sets q->n to the exact count.
wv_status build_query(wv_server_s *S, SQuery *q, const std::vector<uint32_t> &slots) {
  const uint64_t cap = q->n;  // the admission bound
  q->n_cap = cap;
  WV_CHECK(scratch_alloc((void **)&q->d_primes, cap * 8, S->sa));
  uint64_t n = cap;
  if (q->kind == 0) {
    WV_CHECK(sieve_device(q->lo, q->hi, q->d_primes, cap, &n, S->sa));
  } else {
    q->h_primes.assign(1, q->lo);
    WV_CUDA(cudaMemcpyAsync(q->d_primes, q->h_primes.data(), 8, cudaMemcpyHostToDevice, S->sa));
  }
  q->n = n;
  if (n == 0) return WV_OK;
  WV_CHECK(scratch_alloc((void **)&q->d_rb, n * 8, S->sa));
  WV_CHECK(scratch_alloc((void **)&q->d_re, n * 8, S->sa));
  if (q->kind == 0) {
    q->h_primes.resize(n);
    WV_CUDA(cudaMemcpyAsync(q->h_primes.data(), q->d_primes, n * 8, cudaMemcpyDeviceToHost, S->sa));
  }
  WV_CUDA(cudaStreamSynchronize(S->sa));
  q->remaining = 0;
  const ResidueConfig qc = query_cfg(S, q);  // the congruences for this query's primes
  const size_t nplans = (size_t)((n + kPlanPrimes - 1) / kPlanPrimes);
  for (size_t i = 0; i < nplans; ++i) {
    SChunk c;
    c.off = (uint32_t)(i * kPlanPrimes);
    c.n = (uint32_t)std::min<uint64_t>(kPlanPrimes, n - c.off);
    c.slot = slots[i];
    q->chunks.push_back(c);
    SChunk &cc = q->chunks.back();
    // upper bounds on the plan's terms per kernel, O(n): a row holds at most
    // (y - x) p + 1 terms; the planner's exact counts replace them below
    double tb[2] = {0, 0};
    terms_linear(q->h_primes.data() + cc.off, cc.n, qc, tb);
    WV_CHECK(plan_build(q->d_primes + cc.off, cc.n, qc, &cc.plan, S->sa, tb));
    WV_CHECK(plan_totals(&cc.plan, S->sa));
    Plan *dst = (Plan *)((char *)S->d_plans + (size_t)cc.slot * plan_struct_bytes());
    WV_CHECK(plan_upload(&cc.plan, dst, S->sa));
    cc.hi31 = cc.plan.split;
    cc.hi64 = cc.plan.total;
    double t31 = cc.plan.terms[0], t64 = cc.plan.terms[1];
    if (t31 < 0) terms_host(q->h_primes.data() + cc.off, cc.n, qc, &t31, &t64);  // warp tiles
    cc.tpt31 = cc.plan.split ? t31 / cc.plan.split : 1.0;
    cc.tpt64 = (cc.plan.total > cc.plan.split) ? t64 / (cc.plan.total - cc.plan.split) : 1.0;
    q->remaining += t31 + kWideWeight * t64;
  }
  WV_CUDA(cudaStreamSynchronize(S->sa));  // plans visible before the worker sees the query
  return WV_OK;
}

void fail_query(wv_server_s *S, SQuery *q, wv_status st) {
  q->state = 3;
  q->status = st;
  q->err = wv_last_error();
  q->t_done = S->now();
}

// Admission thread.  Among the pending queries (the oldest kAdmitScan), the
// one needing the least device memory that fits the budget, the active-query
// limit and the plan slots goes first (shortest job first: a single prime is
// not held up behind the planning of large ranges); a query pending for more
// than kAdmitAge seconds goes before any other, and while it does not fit
// nothing else is admitted, so large queries cannot starve.  A query is
// always admitted when nothing is active.
void admitter_main(wv_server_s *S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<SQuery *> cand;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_admit.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->stop) return;
      const size_t m = std::min(S->pending.size(), kAdmitScan);
      cand.assign(S->pending.begin(), S->pending.begin() + m);
    }
    // device needs from an upper bound on the prime count (no device work)
    for (SQuery *q : cand) {
      if (q->counted) continue;
      const uint64_t n = q->kind == 0 ? prime_count_bound(q->lo, q->hi) : 1;
      q->count_status = WV_OK;
      if ((n + kPlanPrimes - 1) / kPlanPrimes > kMaxPlans) {
        q->count_status = WV_ENOMEM;
        q->err = "query needs more plan slots than the server has";
      }
      q->n = n;
      q->bytes = query_bytes(S, q, n);
      q->counted = true;
    }
    SQuery *q = nullptr;
    std::vector<uint32_t> slots;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) return;
      auto fits = [&](const SQuery *c) {
        const size_t nplans = (size_t)((c->n + kPlanPrimes - 1) / kPlanPrimes);
        const bool alone = S->active.empty();
        return (alone || (S->bytes_in_use + c->bytes <= S->cfg.mem_budget &&
                          S->active.size() < S->cfg.max_active)) &&
               nplans <= S->free_slots.size();
      };
      const double t = S->now();
      for (SQuery *c : cand)
        if (c->count_status != WV_OK) {
          q = c;
          break;
        }
      if (!q && t - cand.front()->t_submit > kAdmitAge) {
        if (fits(cand.front())) q = cand.front();  // the aged head, or nothing
      } else if (!q) {
        for (SQuery *c : cand)
          if ((!q || c->bytes < q->bytes) && fits(c)) q = c;
      }
      if (!q) {
        // a query finished or arrived; re-check the age of the head now and then
        S->cv_admit.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      S->pending.erase(std::find(S->pending.begin(), S->pending.end(), q));
      if (q->count_status != WV_OK) {
        q->status = q->count_status;
        q->state = 3;
        q->t_done = S->now();
        S->cv_done.notify_all();
        continue;
      }
      q->t_admit = S->now();
      S->bytes_in_use += q->bytes;
      const size_t nplans = (size_t)((q->n + kPlanPrimes - 1) / kPlanPrimes);
      for (size_t i = 0; i < nplans; ++i) {
        slots.push_back(S->free_slots.back());
        S->free_slots.pop_back();
      }
    }
    clear_error();
    wv_status st = build_query(S, q, slots);
    if (st != WV_OK) {
      fail_query(S, q, st);
      const size_t used = q->chunks.size();  // slots of built chunks go back with them
      release_device(S, q, S->sa);
      std::lock_guard<std::mutex> lk(S->mu);
      for (size_t i = used; i < slots.size(); ++i) S->free_slots.push_back(slots[i]);
      S->bytes_in_use -= std::min(S->bytes_in_use, q->bytes);
      S->cv_done.notify_all();
      continue;
    }
    // exact needs now that the range is sieved: give back the rest (the
    // prime buffer keeps its bound-sized allocation)
    if (q->n == 0) release_device(S, q, S->sa);
    const size_t exact = q->n ? query_bytes(S, q, q->n) + (q->n_cap - q->n) * 8 : 0;
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = q->chunks.size(); i < slots.size(); ++i) S->free_slots.push_back(slots[i]);
    if (exact < q->bytes) {
      S->bytes_in_use -= std::min(S->bytes_in_use, q->bytes - exact);
      q->bytes = exact;
      S->cv_admit.notify_all();
    }
    if (q->n == 0) {
      q->state = 2;
      q->t_done = S->now();
      S->cv_done.notify_all();
      continue;
    }
    q->state = 1;
    S->active.push_back(q);
    S->peak_active = std::max<uint32_t>(S->peak_active, (uint32_t)S->active.size());
    S->cv_work.notify_one();
  }
}

// Copy a finished query's residues to the host and release its device memory.
void finish_query(wv_server_s *S, SQuery *q) {
  q->h_rb.resize(q->n);
  q->h_re.resize(q->n);
  cudaError_t e = cudaMemcpyAsync(q->h_rb.data(), q->d_rb, q->n * 8, cudaMemcpyDeviceToHost, S->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q->h_re.data(), q->d_re, q->n * 8, cudaMemcpyDeviceToHost, S->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
  release_device(S, q, S->st);
  if (e != cudaSuccess) {
    fail_query(S, q, cuda_fail(e, "serve: results"));
    return;
  }
  uint64_t h = 0;
  for (size_t i = 0; i < q->n; ++i) h += (q->h_rb[i] == 0 || q->h_re[i] == 0) ? 1 : 0;
  q->n_hits = h;
  q->t_done = S->now();
  q->state = 2;
}

// One epoch's launches on stream es (items already copied to d / h).
wv_status launch_epoch(wv_server_s *S, int b, const std::vector<EpochItem> &items, EpochItem *h,
                       EpochItem *d, uint32_t tot, cudaStream_t es) {
  const int form = S->cfg.epoch_form;
  if (form == 2) return epoch_launch_tiles(d, (uint32_t)items.size(), tot, S->d_plans, S->rcfg, es);
  if (form <= 1)  // the default: one launch (and one tail) per epoch
    return epoch_launch_mixed(d, (uint32_t)items.size(), tot, S->d_plans, S->d_counter + 2 * b,
                              S->rcfg, S->sms, kReserveBlocks, es);
  // form 3: the items of each path as their own list (h is pinned host memory
  // of 2 kMaxPlans items; the 32-bit items first, then the 64-bit ones)
  uint32_t n31 = 0, t31 = 0, t64 = 0;
  for (const EpochItem &it : items)
    if (!(it.plan >> 31)) {
      h[n31] = it;
      h[n31].prefix = t31;
      t31 += it.count;
      ++n31;
    }
  uint32_t n64 = 0;
  for (const EpochItem &it : items)
    if (it.plan >> 31) {
      EpochItem x = it;
      x.plan &= 0x7fffffffu;
      x.prefix = t64;
      t64 += it.count;
      h[n31 + n64++] = x;
    }
  WV_CUDA(cudaMemcpyAsync(d, h, items.size() * sizeof(EpochItem), cudaMemcpyHostToDevice, es));
  if (n31)
    WV_CHECK(epoch_launch(false, d, n31, t31, S->d_plans, S->d_counter + 2 * b, S->rcfg, S->sms,
                          kReserveBlocks, es));
  if (n64)
    WV_CHECK(epoch_launch(true, d + n31, n64, t64, S->d_plans, S->d_counter + 2 * b + 1, S->rcfg,
                          S->sms, kReserveBlocks, es));
  return WV_OK;
}

// Worker thread: epochs, retirement, finalisation.
void worker_main(wv_server_s *S) {
  cudaSetDevice(S->device);
  int64_t epoch_k = 0, completed = -1;
  std::deque<int64_t> inflight;
  for (;;) {
    std::vector<SQuery *> act;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->active.empty() || !inflight.empty(); });
      if (S->stop) {
        lk.unlock();
        for (int b = 0; b < 2; ++b) cudaStreamSynchronize(S->se[b]);
        return;
      }
      act = S->active;
    }
    clear_error();
    // ---- launch one epoch (at most two in flight), smallest remaining work first
    std::sort(act.begin(), act.end(),
              [](const SQuery *a, const SQuery *b) { return a->remaining < b->remaining; });
    wv_status st = WV_OK;
    bool launched = false;
    if (inflight.size() < 2) {
      // epoch size: short while a small query waits (its latency is at least
      // one epoch), up to the configured size when only large work remains
      double budget = S->cfg.epoch_terms;
      for (SQuery *q : act)
        if (q->remaining > 0) {
          budget = std::min(budget, std::max(kMinEpochTerms, 2.0 * q->remaining));
          break;
        }
      std::vector<EpochItem> items;
      uint32_t tot = 0;
      const int64_t k = epoch_k;
      for (SQuery *q : act) {
        for (SChunk &c : q->chunks) {
          if (budget <= 0 || items.size() + 2 > 2 * kMaxPlans) break;
          if (c.hi31 > 0) {
            uint32_t kk = (uint32_t)std::min<double>(c.hi31, std::max(1.0, budget / c.tpt31));
            items.push_back({c.slot, c.hi31 - kk, kk, tot});
            tot += kk;
            c.hi31 -= kk;
            budget -= kk * c.tpt31;
            q->remaining -= kk * c.tpt31;
            c.last_epoch = k;
          }
          if (budget > 0 && c.hi64 > c.plan.split) {
            const uint32_t avail = c.hi64 - c.plan.split;
            uint32_t kk = (uint32_t)std::min<double>(avail, std::max(1.0, budget / (kWideWeight * c.tpt64)));
            items.push_back({c.slot | 0x80000000u, c.hi64 - kk, kk, tot});
            tot += kk;
            c.hi64 -= kk;
            budget -= kWideWeight * kk * c.tpt64;
            q->remaining -= kWideWeight * kk * c.tpt64;
            c.last_epoch = k;
          }
        }
        if (budget <= 0) break;
      }
      if (!items.empty()) {
        const int b = (int)(k & 1);
        cudaStream_t es = S->se[b];
        // this half of the item buffers was used by epoch k-2, which has retired
        EpochItem *h = S->h_items + (size_t)b * 2 * kMaxPlans;
        EpochItem *d = S->d_items + (size_t)b * 2 * kMaxPlans;
        std::copy(items.begin(), items.end(), h);
        cudaError_t e = cudaMemcpyAsync(d, h, items.size() * sizeof(EpochItem), cudaMemcpyHostToDevice, es);
        if (e != cudaSuccess) st = cuda_fail(e, "serve: items");
        if (st == WV_OK) st = launch_epoch(S, b, items, h, d, tot, es);
        if (st == WV_OK && (e = cudaEventRecord(S->ev[b], es)) != cudaSuccess)
          st = cuda_fail(e, "serve: event");
        inflight.push_back(k);
        epoch_k++;
        launched = true;
        std::lock_guard<std::mutex> lk(S->mu);
        S->epochs++;
        S->tiles += tot;
      }
    }
    // ---- retire the oldest epoch once two are in flight (or nothing new started)
    if (st == WV_OK && !inflight.empty() && (inflight.size() >= 2 || !launched)) {
      const int64_t done_k = inflight.front();
      inflight.pop_front();
      cudaError_t e = cudaEventSynchronize(S->ev[done_k & 1]);
      if (e != cudaSuccess) st = cuda_fail(e, "serve: epoch");
      else completed = done_k;
    }
    // ---- finalise plans whose tiles have all run; finish complete queries
    std::vector<SQuery *> finished;
    for (SQuery *q : act) {
      if (st != WV_OK) {
        for (int b = 0; b < 2; ++b) cudaStreamSynchronize(S->se[b]);
        release_device(S, q, S->st);
        fail_query(S, q, st);
        finished.push_back(q);
        continue;
      }
      bool all = true;
      for (SChunk &c : q->chunks) {
        if (!c.finalized && c.hi31 == 0 && c.hi64 == c.plan.split && c.last_epoch <= completed) {
          wv_status s2 = plan_finalize(&c.plan, q->d_rb + c.off, q->d_re + c.off, S->st);
          if (s2 != WV_OK) st = s2;
          c.finalized = true;
        }
        all = all && c.finalized;
      }
      if (all) {
        finish_query(S, q);
        finished.push_back(q);
      }
    }
    if (!finished.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      for (SQuery *q : finished) {
        S->active.erase(std::remove(S->active.begin(), S->active.end(), q), S->active.end());
        S->bytes_in_use -= std::min(S->bytes_in_use, q->bytes);
      }
      S->cv_done.notify_all();
      S->cv_admit.notify_all();
    }
  }
}

void fill_info(const SQuery *q, wv_query_info *info) {
  info->id = q->id;
  info->kind = q->kind;
  info->state = q->state;
  info->status = q->status;
  info->n_primes = q->n;
  info->n_hits = q->n_hits;
  info->t_submit = q->t_submit;
  info->t_admit = q->t_admit;
  info->t_done = q->t_done;
}

}  // namespace

extern "C" {

wv_status wv_server_create(const wv_server_config *cfg, wv_server *out) {
  clear_error();
  if (!out) return set_error(WV_EINVAL, "out is NULL");
  *out = nullptr;
  wv_server_s *S = new wv_server_s();
  if (cfg) S->cfg = *cfg;
  if (S->cfg.mem_budget == 0) S->cfg.mem_budget = (size_t)64 << 30;
  if (S->cfg.max_active == 0) S->cfg.max_active = 256;
  if (S->cfg.epoch_terms <= 0) S->cfg.epoch_terms = 4e10;
  int dev = S->cfg.device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
      delete S;
      return cuda_fail(e, "wv_server_create");
    }
  }
  S->device = dev;
  cudaError_t e = cudaSetDevice(dev);
  DeviceState *ds = nullptr;
  wv_status st = (e == cudaSuccess) ? device_state(&ds) : cuda_fail(e, "cudaSetDevice");
  if (st == WV_OK) {
    S->sms = ds->sms;
    st = resolve_config(nullptr, true, true, &S->rcfg);  // on error, S is freed below
    // small epoch blocks (one warp by default): a warp that runs out of tiles
    // frees its registers at once for the next epoch, not after its block
    S->rcfg.block = S->cfg.epoch_block > 0 ? S->cfg.epoch_block : kEpochBlock;
    if (S->rcfg.block % 32 || S->rcfg.block > 256) st = set_error(WV_EINVAL, "epoch_block must be 32..256, a multiple of 32");
    if (S->cfg.epoch_form < 0 || S->cfg.epoch_form > 3) st = set_error(WV_EINVAL, "epoch_form must be 0..3");
    if (S->cfg.piece_log2 != 0 && (S->cfg.piece_log2 < 12 || S->cfg.piece_log2 > 24))
      st = set_error(WV_EINVAL, "piece_log2 must be 0 or 12..24");
    else if (S->cfg.piece_log2)
      S->rcfg.epoch_piece_max = 1ull << S->cfg.piece_log2;
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    // admission and finalisation go first whenever SMs free up
    e = cudaStreamCreateWithPriority(&S->st, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S->sa, cudaStreamNonBlocking, hi_prio);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&S->se[b], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&S->d_plans, kMaxPlans * plan_struct_bytes());
    if (e == cudaSuccess) e = cudaMalloc(&S->d_items, 4 * kMaxPlans * sizeof(EpochItem));
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_items, 4 * kMaxPlans * sizeof(EpochItem));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_counter, 4 * sizeof(uint32_t));
    if (e != cudaSuccess) st = cuda_fail(e, "wv_server_create");
  }
  if (st != WV_OK) {
    if (S->st) cudaStreamDestroy(S->st);
    if (S->sa) cudaStreamDestroy(S->sa);
    for (int b = 0; b < 2; ++b) {
      if (S->se[b]) cudaStreamDestroy(S->se[b]);
      if (S->ev[b]) cudaEventDestroy(S->ev[b]);
    }
    cudaFree(S->d_plans);
    cudaFree(S->d_items);
    cudaFreeHost(S->h_items);
    cudaFree(S->d_counter);
    delete S;
    return st;
  }
  for (uint32_t i = 0; i < kMaxPlans; ++i) S->free_slots.push_back(kMaxPlans - 1 - i);
  S->t0 = std::chrono::steady_clock::now();
  S->worker = std::thread(worker_main, S);
  S->admitter = std::thread(admitter_main, S);
  *out = S;
  return WV_OK;
}

static wv_status submit(wv_server s, int kind, uint64_t lo, uint64_t hi, uint64_t *id) {
  clear_error();
  if (!s || !id) return set_error(WV_EINVAL, "invalid server or id pointer");
  SQuery *q = new SQuery();
  q->kind = kind;
  q->lo = lo;
  q->hi = hi;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete q;
    return set_error(WV_ECANCELLED, "server is stopping");
  }
  q->id = s->next_id++;
  q->t_submit = s->now();
  s->queries[q->id] = q;
  s->pending.push_back(q);
  *id = q->id;
  s->cv_admit.notify_all();
  return WV_OK;
}

wv_status wv_server_submit_range(wv_server s, uint64_t lo, uint64_t hi, uint64_t *id) {
  if (hi > WV_P_MAX || lo > hi) {
    clear_error();
    return set_error(WV_EINVAL, "range [%llu, %llu) invalid", (unsigned long long)lo,
                     (unsigned long long)hi);
  }
  return submit(s, 0, lo < 5 ? 5 : lo, hi < 5 ? 5 : hi, id);
}

wv_status wv_server_submit_prime(wv_server s, uint64_t p, uint64_t *id) {
  if (p < 5 || p >= WV_P_MAX || !(p & 1)) {
    clear_error();
    return set_error(WV_EINVAL, "p=%llu outside 5 <= p < 2^37 or even", (unsigned long long)p);
  }
  return submit(s, 1, p, p + 1, id);
}

wv_status wv_server_wait(wv_server s, uint64_t id, double timeout_s, wv_query_info *info) {
  clear_error();
  if (!s) return set_error(WV_EINVAL, "invalid server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->queries.find(id);
  if (it == s->queries.end()) return set_error(WV_EINVAL, "unknown query %llu", (unsigned long long)id);
  SQuery *q = it->second;
  auto done = [&] { return q->state >= 2; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
    if (info) fill_info(q, info);
    return set_error(WV_ETIMEOUT, "query %llu not finished", (unsigned long long)id);
  }
  if (info) fill_info(q, info);
  if (q->state == 3) return set_error(q->status, "%s", q->err.c_str());
  if (q->state == 4) return set_error(WV_ECANCELLED, "query cancelled");
  return WV_OK;
}

wv_status wv_server_query(wv_server s, uint64_t id, wv_query_info *info) {
  clear_error();
  if (!s || !info) return set_error(WV_EINVAL, "invalid arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->queries.find(id);
  if (it == s->queries.end()) return set_error(WV_EINVAL, "unknown query %llu", (unsigned long long)id);
  fill_info(it->second, info);
  return WV_OK;
}

wv_status wv_server_result(wv_server s, uint64_t id, uint64_t *h_primes, uint64_t *h_res_b,
                           uint64_t *h_res_e, size_t cap, size_t *n) {
  clear_error();
  if (!s || !n) return set_error(WV_EINVAL, "invalid arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->queries.find(id);
  if (it == s->queries.end()) return set_error(WV_EINVAL, "unknown query %llu", (unsigned long long)id);
  SQuery *q = it->second;
  if (q->state != 2) return set_error(WV_EBUSY, "query %llu is not done", (unsigned long long)id);
  *n = q->n;
  const size_t m = std::min(cap, q->n);
  if (h_primes) std::copy(q->h_primes.begin(), q->h_primes.begin() + m, h_primes);
  if (h_res_b) std::copy(q->h_rb.begin(), q->h_rb.begin() + m, h_res_b);
  if (h_res_e) std::copy(q->h_re.begin(), q->h_re.begin() + m, h_res_e);
  if (cap < q->n) return set_error(WV_ERANGE, "%zu primes, capacity %zu", q->n, cap);
  return WV_OK;
}

wv_status wv_server_release(wv_server s, uint64_t id) {
  clear_error();
  if (!s) return set_error(WV_EINVAL, "invalid server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->queries.find(id);
  if (it == s->queries.end()) return WV_OK;
  if (it->second->state < 2) return set_error(WV_EBUSY, "query %llu still running", (unsigned long long)id);
  delete it->second;
  s->queries.erase(it);
  return WV_OK;
}

wv_status wv_server_stats(wv_server s, uint64_t *epochs, uint64_t *tiles, size_t *bytes_in_use,
                          uint32_t *peak_active) {
  clear_error();
  if (!s) return set_error(WV_EINVAL, "invalid server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (epochs) *epochs = s->epochs;
  if (tiles) *tiles = s->tiles;
  if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
  if (peak_active) *peak_active = s->peak_active;
  return WV_OK;
}

wv_status wv_server_destroy(wv_server s) {
  clear_error();
  if (!s) return WV_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
    s->cv_admit.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->admitter.joinable()) s->admitter.join();
  cudaSetDevice(s->device);
  for (int b = 0; b < 2; ++b) cudaStreamSynchronize(s->se[b]);
  cudaStreamSynchronize(s->sa);
  for (auto &kv : s->queries) {
    SQuery *q = kv.second;
    if (q->state < 2) {
      release_device(s, q, s->st);
      q->state = 4;
    }
  }
  cudaStreamSynchronize(s->st);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_done.notify_all();
  }
  for (auto &kv : s->queries) delete kv.second;
  s->queries.clear();
  cudaFree(s->d_plans);
  cudaFree(s->d_items);
  cudaFreeHost(s->h_items);
  cudaFree(s->d_counter);
  cudaStreamDestroy(s->st);
  cudaStreamDestroy(s->sa);
  for (int b = 0; b < 2; ++b) {
    cudaStreamDestroy(s->se[b]);
    cudaEventDestroy(s->ev[b]);
  }
  delete s;
  return WV_OK;
}

}  // extern "C"
