// wv_registry.cu -- every congruence the library can run, in one table.
//
// Built-in congruences (the transcribed tables of Sec. 3 and Sec. 5,
// wv_tables.h), the generated ones (greedy search over Prop. 2.1,
// wv_tables_gen.h) and the general-index forms (wv_residues_general) are
// brought to one representation: a row is an interval (xn/xd, yn/yd) with a
// coefficient sum_k c_k d_k^t, stored as terms (c_k, index of d_k in the
// congruence's list of distinct bases).  A built-in row is the single term
// (coef, d = 1).  The table is built once on the host and uploaded once per
// device (DeviceState).
#include <mutex>
#include <string>
#include <vector>

#include "wv_arith.cuh"
#include "wv_internal.h"
#include "wv_tables.h"
#include "wv_tables_gen.h"

namespace wv {

namespace {

struct Registry {
  std::vector<CongView> views;  // built-in, generated, then the two general forms
  std::vector<uint32_t> rows;   // 6 words per row: xn, xd, yn, yd, first term, number of terms
  std::vector<int64_t> tc;
  std::vector<uint16_t> td;
  std::vector<uint64_t> dist;
  int n_public = 0;             // built-in + generated
};

Registry build_registry() {
  Registry R;
  auto begin = [&](const char *name, int kind, int nrows, int64_t lhs) {
    CongView v;
    v.name = name;
    v.kind = kind;
    v.nrows = nrows;
    v.lhs = lhs;
    v.row0 = (uint32_t)(R.rows.size() / 6);
    v.dist0 = (uint32_t)R.dist.size();
    v.ndist = 0;
    return v;
  };
  for (int i = 0; i < kWvNumCongruences; ++i) {
    const WvCongruence &c = kWvCongruences[i];
    CongView v = begin(c.name, c.kind, c.nrows, c.lhs);
    R.dist.push_back(1);
    v.ndist = 1;
    for (int j = 0; j < c.nrows; ++j) {
      const WvRow &w = kWvRows[c.row_offset + j];
      R.rows.insert(R.rows.end(), {w.xn, w.xd, w.yn, w.yd, (uint32_t)R.tc.size(), 1u});
      R.tc.push_back(w.coef);
      R.td.push_back(0);
    }
    R.views.push_back(v);
  }
  for (int i = 0; i < kWvNumGenTables; ++i) {
    const WvGenTable &g = kWvGenTables[i];
    CongView v = begin(g.name, g.kind, g.nrows, g.lhs);
    for (uint32_t k = 0; k < g.ndist; ++k) R.dist.push_back(kWvGenDist[g.dist0 + k]);
    v.ndist = g.ndist;
    for (int j = 0; j < g.nrows; ++j) {
      const uint32_t *w = kWvGenRows[g.row0 + j];
      R.rows.insert(R.rows.end(), {w[0], w[1], w[2], w[3], (uint32_t)R.tc.size(), w[5]});
      for (uint32_t k = 0; k < w[5]; ++k) {
        R.tc.push_back(kWvGenTermC[w[4] + k]);
        R.td.push_back(kWvGenTermD[w[4] + k]);
      }
    }
    R.views.push_back(v);
  }
  R.n_public = (int)R.views.size();
  for (int kind = 0; kind < 2; ++kind) {
    const WvGenCongruence &g = kWvGeneral[kind];
    CongView v = begin(g.name, g.kind, g.nrows, 0);
    std::vector<uint64_t> ds;
    for (int j = 0; j < g.nrows; ++j)
      for (int k = 0; k < 3; ++k)
        if (g.rows[j].c[k]) {
          bool have = false;
          for (uint64_t d : ds) have = have || d == g.rows[j].d[k];
          if (!have) ds.push_back(g.rows[j].d[k]);
        }
    for (uint64_t d : ds) R.dist.push_back(d);
    v.ndist = (uint32_t)ds.size();
    for (int j = 0; j < g.nrows; ++j) {
      const WvGenRow &w = g.rows[j];
      uint32_t nt = 0;
      const uint32_t t0 = (uint32_t)R.tc.size();
      for (int k = 0; k < 3; ++k)
        if (w.c[k]) {
          R.tc.push_back(w.c[k]);
          uint16_t idx = 0;
          for (size_t q = 0; q < ds.size(); ++q)
            if (ds[q] == w.d[k]) idx = (uint16_t)q;
          R.td.push_back(idx);
          ++nt;
        }
      R.rows.insert(R.rows.end(), {w.xn, w.xd, w.yn, w.yd, t0, nt});
    }
    R.views.push_back(v);
  }
  return R;
}

const Registry &registry() {
  static const Registry R = build_registry();
  return R;
}

}  // namespace

int cong_count() { return registry().n_public; }

static int id_of(const char *name, int fallback) {
  for (int i = 0; i < cong_count(); ++i)
    if (std::string(cong_view(i).name) == name) return i;
  return fallback;
}

// The default for a prime list whose range is not known: the paper's BB30 and
// EE33, good at every p (the generated congruences win only where their
// shorter sums are still long, see cong_for_range).
int cong_default(int kind) { return kind == 0 ? kWvDefaultB : kWvDefaultE; }

// The congruences for primes below `hi` (the paper also switches congruences
// with the size of p, Sec. 3 "Method for primes p < 6e10").  Measured on
// GB300 with lane chains, for each kind alone, over windows of primes from
// 1e5 to 1e11: with lane chains every congruence runs at the kernel's own
// rate once its sums are a few thousand terms long, so the cheaper ones
// (more sums) win as p grows: BB2244 + EE2004 from 1.5e8, BB3802 + EE4122
// (about twice the sums, which the planner and finaliser pay per prime)
// from 1.2e9.
void cong_for_range(uint64_t hi, int *cb, int *ce) {
  struct Band {
    uint64_t hi;
    const char *name;
  };
  static const Band bands_b[] = {{5000000ull, "BB30"},      {20000000ull, "BB249"},
                                 {50000000ull, "BB476"},    {150000000ull, "BB1115"},
                                 {1200000000ull, "BB2244"}, {~0ull, "BB3802"}};
  static const Band bands_e[] = {{3000000ull, "EE33"},      {20000000ull, "EE200"},
                                 {50000000ull, "EE404"},    {150000000ull, "EE967"},
                                 {1200000000ull, "EE2004"}, {~0ull, "EE4122"}};
  for (const Band &bd : bands_b)
    if (hi <= bd.hi) {
      *cb = id_of(bd.name, kWvDefaultB);
      break;
    }
  for (const Band &bd : bands_e)
    if (hi <= bd.hi) {
      *ce = id_of(bd.name, kWvDefaultE);
      break;
    }
}

int cong_general_id(int kind) { return registry().n_public + kind; }
const CongView &cong_view(int id) { return registry().views[id]; }
const uint32_t *cong_row(uint32_t r) { return &registry().rows[6 * (size_t)r]; }
const int64_t *cong_tc() { return registry().tc.data(); }
const uint16_t *cong_td() { return registry().td.data(); }
const uint64_t *cong_dist() { return registry().dist.data(); }

wv_status cong_upload(DeviceState *d) {
  const Registry &R = registry();
  for (const CongView &v : R.views)
    if (v.ndist > 512) return set_error(WV_EINVAL, "congruence %s: %u bases (max 512)", v.name, v.ndist);
  WV_CUDA(cudaMalloc(&d->cg_rows, R.rows.size() * sizeof(uint32_t)));
  WV_CUDA(cudaMalloc(&d->cg_tc, R.tc.size() * sizeof(int64_t)));
  WV_CUDA(cudaMalloc(&d->cg_td, R.td.size() * sizeof(uint16_t)));
  WV_CUDA(cudaMalloc(&d->cg_dist, R.dist.size() * sizeof(uint64_t)));
  WV_CUDA(cudaMemcpy(d->cg_rows, R.rows.data(), R.rows.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  WV_CUDA(cudaMemcpy(d->cg_tc, R.tc.data(), R.tc.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  WV_CUDA(cudaMemcpy(d->cg_td, R.td.data(), R.td.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  WV_CUDA(cudaMemcpy(d->cg_dist, R.dist.data(), R.dist.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
  // copies from pageable memory can return before the data is on the device;
  // a caller's non-blocking stream is not ordered after them
  WV_CUDA(cudaDeviceSynchronize());
  return WV_OK;
}

}  // namespace wv

extern "C" int wv_congruence_default(int kind) { return wv::cong_default(kind); }

extern "C" void wv_congruence_for_range(uint64_t lo, uint64_t hi, int *cong_b, int *cong_e) {
  (void)lo;
  int b = 0, e = 0;
  wv::cong_for_range(hi, &b, &e);
  if (cong_b) *cong_b = b;
  if (cong_e) *cong_e = e;
}

namespace wv {

uint64_t cong_row_terms(uint32_t r, uint64_t p) {
  const uint32_t *w = cong_row(r);
  const uint64_t lo = floor_frac_times(w[0], w[1], p) + 1;
  const uint64_t hi = floor_frac_times(w[2], w[3], p) + 1;
  return hi > lo ? hi - lo : 0;
}

}  // namespace wv
