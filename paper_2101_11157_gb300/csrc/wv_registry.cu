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

// The library's default congruences: generated ones, BB249 (cost p/38.2,
// from B30) and EE404 (cost p/29.8, from E33).  Against BB30 + EE33 they cut
// the terms per prime by 32 %; more sums make the tiles shorter and their
// per-tile work outweighs the saving at p ~ 1e9 (measured).
int cong_default(int kind) {
  static const int ids[2] = {[] {
                               for (int i = 0; i < cong_count(); ++i)
                                 if (std::string(cong_view(i).name) == "BB249") return i;
                               return (int)kWvDefaultB;
                             }(),
                             [] {
                               for (int i = 0; i < cong_count(); ++i)
                                 if (std::string(cong_view(i).name) == "EE404") return i;
                               return (int)kWvDefaultE;
                             }()};
  return ids[kind ? 1 : 0];
}
int cong_general_id(int kind) { return registry().n_public + kind; }
const CongView &cong_view(int id) { return registry().views[id]; }
const uint32_t *cong_row(uint32_t r) { return &registry().rows[6 * (size_t)r]; }
const int64_t *cong_tc() { return registry().tc.data(); }
const uint16_t *cong_td() { return registry().td.data(); }
const uint64_t *cong_dist() { return registry().dist.data(); }

wv_status cong_upload(DeviceState *d) {
  const Registry &R = registry();
  WV_CUDA(cudaMalloc(&d->cg_rows, R.rows.size() * sizeof(uint32_t)));
  WV_CUDA(cudaMalloc(&d->cg_tc, R.tc.size() * sizeof(int64_t)));
  WV_CUDA(cudaMalloc(&d->cg_td, R.td.size() * sizeof(uint16_t)));
  WV_CUDA(cudaMalloc(&d->cg_dist, R.dist.size() * sizeof(uint64_t)));
  WV_CUDA(cudaMemcpy(d->cg_rows, R.rows.data(), R.rows.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  WV_CUDA(cudaMemcpy(d->cg_tc, R.tc.data(), R.tc.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  WV_CUDA(cudaMemcpy(d->cg_td, R.td.data(), R.td.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  WV_CUDA(cudaMemcpy(d->cg_dist, R.dist.data(), R.dist.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
  return WV_OK;
}

}  // namespace wv

extern "C" int wv_congruence_default(int kind) { return wv::cong_default(kind); }

namespace wv {

uint64_t cong_row_terms(uint32_t r, uint64_t p) {
  const uint32_t *w = cong_row(r);
  const uint64_t lo = (uint64_t)w[0] * p / w[1] + 1;
  const uint64_t hi = (uint64_t)w[2] * p / w[3] + 1;
  return hi > lo ? hi - lo : 0;
}

}  // namespace wv
