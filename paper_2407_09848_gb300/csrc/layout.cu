// Host-side layout planning (see layout.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <functional>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "host_check.h"
#include "layout.h"

namespace amgps {
namespace {

int64_t floor_to(int64_t x, int64_t a) { return x >= 0 ? x / a * a : -((-x + a - 1) / a) * a; }
int64_t ceil_to(int64_t x, int64_t a) { return -floor_to(-x, a); }

}  // namespace

int parallel_threads(int64_t count) {
  if (count < 4096) return 1;
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hw == 0 ? 1u : hw, 32u));
}

void parallel_for(int64_t count, const std::function<void(int64_t, int)>& f) {
  const int nt = parallel_threads(count);
  if (nt == 1) {
    for (int64_t i = 0; i < count; ++i) f(i, 0);
    return;
  }
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> errs(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      try {
        const int64_t i0 = count * t / nt, i1 = count * (t + 1) / nt;
        for (int64_t i = i0; i < i1; ++i) f(i, t);
      } catch (...) {
        errs[t] = std::current_exception();
      }
    });
  for (auto& x : th) x.join();
  for (auto& e : errs)
    if (e) std::rethrow_exception(e);
}

void validate_csr(const amgps_csr& A, const char* what, bool square) {
  const std::string w(what);
  REQ(A.rowptr && A.col && A.val, AMGPS_E_ARG, w + ": null array");
  REQ(A.n_rows >= 1 && A.n_cols >= 1, AMGPS_E_ARG, w + ": empty matrix");
  REQ(A.n_rows < (int64_t(1) << 31) && A.n_cols < (int64_t(1) << 31), AMGPS_E_ARG,
      w + ": dimension exceeds int32");
  REQ(!square || A.n_rows == A.n_cols, AMGPS_E_ARG, w + ": not square");
  REQ(A.rowptr[0] == 0 && A.rowptr[A.n_rows] == A.nnz, AMGPS_E_ARG, w + ": bad rowptr ends");
  parallel_for(A.n_rows, [&](int64_t i, int) {
    REQ(A.rowptr[i + 1] >= A.rowptr[i], AMGPS_E_ARG, w + ": rowptr not monotone");
  });
  // rowptr is monotone from 0 to nnz, so the rows cover every entry once
  parallel_for(A.n_rows, [&](int64_t i, int) {
    for (int e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      REQ(A.col[e] >= 0 && A.col[e] < A.n_cols, AMGPS_E_ARG, w + ": column index out of range");
      REQ(std::isfinite(A.val[e]), AMGPS_E_ARG, w + ": non-finite value");
    }
  });
}

void require_positive_diagonal(const amgps_csr& A) {
  parallel_for(A.n_rows, [&](int64_t i, int) {
    bool found = false;
    for (int e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (A.col[e] == i) {
        REQ(A.val[e] > 0.0, AMGPS_E_NOT_SPD, "non-positive diagonal entry");
        found = true;
      }
    REQ(found, AMGPS_E_NOT_SPD, "missing diagonal entry");
  });
}

// Warps per slice for the split kernels (measured on the 256^3
// smoothed-aggregation levels): 1 while rows average under 24 stored entries;
// otherwise the larger of a width term (the power of two nearest avg / 32 once
// avg >= 48) and a parallelism term (the power of two at or below
// 24576 / slices, so small levels still field ~24k warps), capped at avg / 8
// entries per warp and kMaxSplit.
int split_for(int64_t stored, int64_t nslices) {
  if (nslices == 0) return 1;
  const double avg = (double)stored / ((double)nslices * kSlice);
  if (avg < 24.0) return 1;
  int g1 = 1;
  if (avg >= 48.0)
    while (g1 < kMaxSplit && 2.0 * g1 <= avg / 32.0 * 1.41421356) g1 *= 2;
  int g2 = 1;
  while (g2 < kMaxSplit && 2.0 * g2 <= 24576.0 / (double)nslices) g2 *= 2;
  int cap = 1;
  while (cap < kMaxSplit && 2.0 * cap <= avg / 8.0) cap *= 2;
  return std::max(1, std::min(std::max(g1, g2), cap));
}



// allow_uniform = false keeps every slice explicit (required for rectangular
// matrices: a uniform slice's padding column row + off may fall outside n_cols)
// Three passes: (1) in parallel, each slice's longest row and its sorted set
// of column offsets; (2) in slice order, the layout decision (a slice whose
// offsets all lie in the previous uniform pattern reuses it, so boundary
// slices keep the interior pattern; else its own offsets if uniform; else
// explicit) and the prefix of value bases; (3) in parallel, the values (and
// explicit columns).  Each slice's output depends on its rows alone, so the
// result does not depend on the thread count.
HostSell build_sell(const amgps_csr& A, bool allow_uniform) {
  HostSell h;
  const int64_t n = A.n_rows;
  h.n = n;
  h.nnz = A.nnz;
  h.nslices = (n + kSlice - 1) / kSlice;
  h.sd.resize(h.nslices);
  std::vector<int32_t> maxlen(h.nslices, 0);
  std::vector<std::vector<int32_t>> own(allow_uniform ? h.nslices : 0);
  parallel_for(h.nslices, [&](int64_t s, int) {
    const int64_t r0 = s * kSlice, r1 = std::min(n, r0 + kSlice);
    int ml = 0;
    for (int64_t r = r0; r < r1; ++r) ml = std::max(ml, A.rowptr[r + 1] - A.rowptr[r]);
    maxlen[s] = ml;
    if (!allow_uniform) return;
    std::vector<int32_t>& o = own[s];
    for (int64_t r = r0; r < r1; ++r)
      for (int e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e)
        o.push_back((int32_t)((int64_t)A.col[e] - r));
    std::sort(o.begin(), o.end());
    o.erase(std::unique(o.begin(), o.end()), o.end());
  });
  std::map<std::vector<int32_t>, int32_t> pats;
  const std::vector<int32_t>* prev = nullptr;
  int32_t prev_ref = -1;
  int64_t vbase = 0;
  for (int64_t s = 0; s < h.nslices; ++s) {
    const int ml = maxlen[s];
    if (allow_uniform && prev_ref >= 0 && (int64_t)prev->size() <= ml + 1 &&
        std::includes(prev->begin(), prev->end(), own[s].begin(), own[s].end())) {
      h.sd[s] = SliceDesc{vbase, (int32_t)prev->size(), prev_ref};
      vbase += (int64_t)prev->size() * kSlice;
      continue;
    }
    const bool uniform = allow_uniform && (int64_t)own[s].size() <= ml + 1 &&
                         (int64_t)own[s].size() <= kUniformMax;
    if (uniform) {
      auto it = pats.find(own[s]);
      int32_t ref;
      if (it == pats.end()) {
        ref = (int32_t)h.off.size();
        h.off.insert(h.off.end(), own[s].begin(), own[s].end());
        it = pats.emplace(own[s], ref).first;
      } else {
        ref = it->second;
      }
      prev = &it->first;
      prev_ref = ref;
      h.sd[s] = SliceDesc{vbase, (int32_t)own[s].size(), ref};
      vbase += (int64_t)own[s].size() * kSlice;
    } else {
      h.sd[s] = SliceDesc{vbase, (int32_t)ml, -1};
      vbase += (int64_t)ml * kSlice;
      h.any_explicit = true;
      h.explicit_entries += (int64_t)ml * kSlice;
    }
  }
  own.clear();
  own.shrink_to_fit();
  h.stored = vbase;
  h.val.assign(vbase, 0.0);
  if (h.any_explicit) h.col.assign(vbase, 0);
  const int nt = parallel_threads(h.nslices);
  std::vector<std::vector<std::pair<int32_t, double>>> rowbufs(nt);
  std::vector<std::vector<uint8_t>> filleds(nt);
  parallel_for(h.nslices, [&](int64_t s, int t) {
    std::vector<std::pair<int32_t, double>>& rowbuf = rowbufs[t];
    std::vector<uint8_t>& filled = filleds[t];
    const SliceDesc d = h.sd[s];
    const int64_t r0 = s * kSlice, r1 = std::min(n, r0 + kSlice);
    for (int64_t r = r0; r < r1; ++r) {
      const int lane = (int)(r - r0);
      if (d.cref >= 0) {
        if ((int)filled.size() < d.w) filled.resize(d.w);
        std::fill(filled.begin(), filled.begin() + d.w, uint8_t(0));
        const int32_t* p = h.off.data() + d.cref;
        for (int e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) {
          const int32_t o = (int32_t)((int64_t)A.col[e] - r);
          const int k = (int)(std::lower_bound(p, p + d.w, o) - p);
          REQ(!filled[k], AMGPS_E_ARG, "duplicate entry in CSR row");
          filled[k] = 1;
          h.val[d.vbase + (int64_t)k * kSlice + lane] = A.val[e];
        }
      } else {
        rowbuf.clear();
        for (int e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) rowbuf.emplace_back(A.col[e], A.val[e]);
        std::sort(rowbuf.begin(), rowbuf.end());
        for (size_t k = 0; k < rowbuf.size(); ++k) {
          REQ(k == 0 || rowbuf[k].first != rowbuf[k - 1].first, AMGPS_E_ARG,
              "duplicate entry in CSR row");
          h.val[d.vbase + (int64_t)k * kSlice + lane] = rowbuf[k].second;
          h.col[d.vbase + (int64_t)k * kSlice + lane] = rowbuf[k].first;
        }
        for (int k = (int)rowbuf.size(); k < d.w; ++k)
          h.col[d.vbase + (int64_t)k * kSlice + lane] = (int32_t)std::min<int64_t>(r, A.n_cols - 1);
      }
    }
  });
  return h;
}

// FP64 -> BF16 round-to-nearest-even taken directly from the double (no
// intermediate FP32 rounding): compare against the neighbouring BF16 values.
uint16_t dbl_to_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  uint32_t base = u & 0xFFFF0000u;
  auto val = [](uint32_t bits) {
    float g;
    std::memcpy(&g, &bits, 4);
    return (double)g;
  };
  uint32_t best = base;
  double bestd = std::fabs(val(base) - x);
  for (int d = -1; d <= 1; d += 2) {
    const uint32_t cand = base + (uint32_t)(d * 0x10000);
    const double cd = std::fabs(val(cand) - x);
    if (std::isfinite(val(cand)) &&
        (cd < bestd || (cd == bestd && ((cand >> 16) & 1u) == 0 && ((best >> 16) & 1u) == 1))) {
      best = cand;
      bestd = cd;
    }
  }
  return (uint16_t)(best >> 16);
}






// Which tiles the TMA-fed step can take, and the shared-memory stage layout for
// them.  A tile qualifies when all its slices share the level's most
// frequent uniform pattern (width <= kTmaMaxW) and every window it copies lies
// inside [0, n).  Every copy range and alignment is re-checked here on the host,
// so the kernel never sees an out-of-bounds or misaligned bulk copy.
HostPlan build_tma_plan(const HostSell& h, size_t vsize, size_t xsize, int smem_budget) {
  HostPlan hp;
  const int64_t n = h.n;
  const int rows = tma_rows(xsize);
  const int64_t ntf = n / rows;
  const int spt = rows / kSlice;
  hp.p.rows = rows;
  auto candidate = [&](int64_t t, int32_t& cref, int& w) {
    const SliceDesc d0 = h.sd[t * spt];
    if (d0.cref < 0 || d0.w < 1 || d0.w > kTmaMaxW) return false;
    for (int i = 1; i < spt; ++i) {
      const SliceDesc d = h.sd[t * spt + i];
      if (d.cref != d0.cref || d.w != d0.w || d.vbase != d0.vbase + (int64_t)i * d0.w * kSlice)
        return false;
    }
    cref = d0.cref;
    w = d0.w;
    return true;
  };
  std::map<int32_t, int64_t> freq;
  std::map<int32_t, int> width;
  for (int64_t t = 0; t < ntf; ++t) {
    int32_t cref;
    int w;
    if (candidate(t, cref, w)) {
      freq[cref]++;
      width[cref] = w;
    }
  }
  std::vector<char> covered(h.nslices, 0);
  auto finish = [&]() {
    for (int64_t s = 0; s < h.nslices; ++s)
      if (!covered[s]) hp.gen.push_back((int32_t)s);
    return hp;
  };
  if (freq.empty()) return finish();
  int32_t dom = freq.begin()->first;
  for (auto& kv : freq)
    if (kv.second > freq[dom]) dom = kv.first;
  TmaPlan& P = hp.p;
  P.w = width[dom];
  const int32_t* off = h.off.data() + dom;
  const int64_t A = 16 / (int64_t)xsize;
  // groups of offsets whose tile-height windows overlap, touch, or leave a
  // gap of at most kTmaMergeSlack elements (copied along)
  int gk[kTmaMaxW];
  int64_t glo[kTmaMaxW], ghi[kTmaMaxW];
  int ng = 0;
  for (int k = 0; k < P.w; ++k) {
    if (ng > 0 && off[k] - ghi[ng - 1] <= rows + kTmaMergeSlack) {
      ghi[ng - 1] = off[k];
    } else {
      glo[ng] = ghi[ng] = off[k];
      ++ng;
    }
    gk[k] = ng - 1;
  }
  if (ng > kTmaMaxGroups) return finish();
  P.ngroups = ng;
  int64_t acc = 0;
  for (int g = 0; g < ng; ++g) {
    const int64_t st = floor_to(glo[g], A), en = ceil_to(ghi[g] + rows, A);
    P.g_start[g] = (int)st;
    P.g_elems[g] = (int)(en - st);
    P.g_smem[g] = (int)acc;
    acc += en - st;
  }
  bool has0 = false;
  for (int k = 0; k < P.w; ++k) {
    P.d[k] = P.g_smem[gk[k]] + (int)(off[k] - P.g_start[gk[k]]);
    if (off[k] == 0) {
      P.d0 = P.d[k];
      has0 = true;
    }
  }
  if (!has0) return finish();
  P.vals_bytes = (int)(P.w * rows * vsize);
  P.vec_bytes = (int)(rows * xsize);
  P.win_bytes = (int)(acc * (int64_t)xsize);
  P.stage_bytes =
      (int)ceil_to(P.vals_bytes + tma_vec_slots(xsize) * P.vec_bytes + P.win_bytes, 128);
  P.nstages = std::min<int>(kTmaMaxStages, (smem_budget - 2 * kTmaMaxStages * 8) / P.stage_bytes);
  P.nstages -= P.nstages % tma_groups(xsize);  // see tma_groups()
  if (P.nstages < 2) {
    P.nstages = 0;
    return finish();
  }
  for (int64_t t = 0; t < ntf; ++t) {
    int32_t cref;
    int w;
    if (!candidate(t, cref, w) || cref != dom) continue;
    const int64_t r0 = t * rows;
    bool ok = true;
    for (int g = 0; g < ng; ++g)
      ok = ok && r0 + P.g_start[g] >= 0 && r0 + P.g_start[g] + P.g_elems[g] <= n;
    if (!ok) continue;
    const int64_t vb = h.sd[t * spt].vbase;
    // host-side proof of every bulk copy of this tile: in bounds and 16-byte aligned
    REQ(vb >= 0 && vb + (int64_t)P.w * rows <= h.stored && (vb * (int64_t)vsize) % 16 == 0,
        AMGPS_E_ARG, "TMA plan: value copy out of range or misaligned");
    REQ(r0 + rows <= n && (r0 * (int64_t)xsize) % 16 == 0, AMGPS_E_ARG,
        "TMA plan: vector copy out of range or misaligned");
    for (int g = 0; g < ng; ++g)
      REQ(((r0 + P.g_start[g]) * (int64_t)xsize) % 16 == 0 &&
              ((int64_t)P.g_elems[g] * (int64_t)xsize) % 16 == 0,
          AMGPS_E_ARG, "TMA plan: window copy misaligned");
    for (int k = 0; k < P.w; ++k)
      REQ(P.d[k] >= 0 && P.d[k] + rows <= acc, AMGPS_E_ARG, "TMA plan: window index out of range");
    hp.tiles.push_back(TmaTile{r0, vb});
    for (int i = 0; i < spt; ++i) covered[t * spt + i] = 1;
  }
  return finish();
}

}  // namespace amgps
