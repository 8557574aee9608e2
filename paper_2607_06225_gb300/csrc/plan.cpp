// plan.cpp -- host planner (see plan.h).
//
// Ordering: pairs are sorted by estimated cost (cells), longest first, so the
// persistent kernels' work queues finish with short pairs and the tail is
// short.  The sort is a counting sort over 64 logarithmic cost buckets (O(n)).
// Waves: with traceback on, every pair needs its 4-bit choices kept until the
// walk; pairs are cut, in cost order, into waves whose traceback fits the
// workspace.  Within a wave, pairs sharing a kernel shape form a group (one
// launch each).
#include "plan.h"

#include <algorithm>
#include <cmath>

#include "k_xdrop_layout.h"

namespace filtr {

int full_rows_per_lane(uint32_t M) { return M <= 256 ? 8 : 16; }

uint64_t full_tb_words(uint32_t M, uint32_t N, int R, const ScoreParams &sp) {
  const int64_t HS = 32 * R;
  int64_t lo = -(int64_t)M - 1, hi = (int64_t)N + 1;
  const bool band = sp.use_band != 0;
  if (band) band_limits(M, N, sp.band, sp.band_literal, &lo, &hi);
  uint64_t w = 0;
  const int64_t ns = (M + HS - 1) / HS;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t jl, jh;
    strip_cols(s * HS, HS, M, N, band, lo, hi, &jl, &jh);
    if (jl > jh) break;
    w += (uint64_t)strip_tb_words(jl, jh, R);
  }
  return w;
}

uint64_t band_cells(uint32_t M, uint32_t N, const ScoreParams &sp) {
  if (!sp.use_band) return (uint64_t)M * N;
  int64_t lo, hi;
  band_limits(M, N, sp.band, sp.band_literal, &lo, &hi);
  // Sum over diagonals d in [lo, hi] of the cells of diagonal d inside the
  // matrix, f(d) = min(M, N - d) - max(0, -d) for 1-M <= d <= N-1.  f is linear
  // between its kinks at d = 0 and d = N - M, so each piece is an arithmetic sum.
  const int64_t Mi = M, Ni = N;
  const int64_t A = std::max<int64_t>(lo, 1 - Mi), B = std::min<int64_t>(hi, Ni - 1);
  if (A > B) return 0;
  auto f = [&](int64_t d) { return std::min<int64_t>(Mi, Ni - d) - std::max<int64_t>(0, -d); };
  const int64_t k1 = std::min<int64_t>(0, Ni - Mi), k2 = std::max<int64_t>(0, Ni - Mi);
  const int64_t cut[4] = {A - 1, std::min(std::max(k1, A - 1), B), std::min(std::max(k2, A - 1), B), B};
  uint64_t c = 0;
  for (int s = 0; s < 3; ++s) {
    const int64_t a = cut[s] + 1, b = cut[s + 1];
    if (b >= a) c += (uint64_t)((f(a) + f(b)) * (b - a + 1) / 2);
  }
  return c;
}

static int cost_bucket(uint64_t cost) {
  if (cost == 0) return 0;
  int b = 0;
  double x = (double)cost;
  b = (int)std::floor(std::log2(x) * 2.0);  // half-octave buckets
  return std::min(63, std::max(0, b));
}

bool make_plan(const PlanInput &in, Plan *P) {
  const ScoreParams &sp = *in.sp;
  const uint32_t n = in.n;
  P->order.clear();
  P->tbl.assign(n, TbLayout{});
  P->stage_off.assign(n, 0);
  P->waves.clear();
  P->trivial.clear();
  P->stage_words = 0;
  P->max_n = P->max_m = 0;
  P->cigar_upper = 0;
  P->cells_estimate = 0;

  std::vector<PairPlan> pp;
  pp.reserve(n);
  for (uint32_t p = 0; p < n; ++p) {
    const uint32_t M = in.q_len[p], N = in.r_len[p];
    P->max_n = std::max<uint64_t>(P->max_n, N);
    P->max_m = std::max<uint64_t>(P->max_m, M);
    P->cigar_upper += (uint64_t)M + N;
    if (sp.traceback) {
      P->stage_off[p] = P->stage_words;
      P->stage_words += (uint64_t)M + N + 1;
    }
    // an empty side leaves no cell to evaluate, except under X-drop, where the
    // gap cells of row 0 / column 0 are themselves subject to the prune test
    if ((M == 0 && N == 0) || ((M == 0 || N == 0) && !sp.use_xdrop)) {
      P->trivial.push_back(p);
      if (sp.traceback) P->tbl[p].valid = 0;
      continue;
    }
    PairPlan x{};
    x.pair = p;
    if (sp.use_xdrop) {
      x.family = FAM_XDROP;
      x.R = (uint8_t)in.xdrop_slots;
      x.warps = (uint8_t)(in.xdrop_warps > 0 ? in.xdrop_warps : 1);
      x.tb_words = sp.traceback ? xd_tb_words(M, N, x.warps, x.R) : 0;
      // the live region is data dependent; its cost is at most the band / matrix
      x.cost = band_cells(M, N, sp);
    } else {
      x.family = FAM_FULL;
      x.R = (uint8_t)full_rows_per_lane(M);
      x.warps = 1;
      x.tb_words = sp.traceback ? full_tb_words(M, N, x.R, sp) : 0;
      x.cost = band_cells(M, N, sp);
    }
    P->cells_estimate += x.cost;
    if (sp.traceback && x.tb_words > in.tb_budget_words) {
      set_error("pair %u needs %llu traceback bytes, more than the workspace allows", p,
                (unsigned long long)(x.tb_words * 4));
      return false;
    }
    pp.push_back(x);
  }

  // counting sort, most expensive bucket first
  std::vector<uint32_t> cnt(64, 0);
  for (auto &x : pp) cnt[63 - cost_bucket(x.cost)]++;
  std::vector<uint32_t> start(64, 0);
  for (int b = 1; b < 64; ++b) start[b] = start[b - 1] + cnt[b - 1];
  std::vector<PairPlan> sorted(pp.size());
  for (auto &x : pp) sorted[start[63 - cost_bucket(x.cost)]++] = x;

  // waves
  const uint64_t budget = sp.traceback ? in.tb_budget_words : ~0ull;
  size_t i = 0;
  while (i < sorted.size()) {
    size_t j = i;
    uint64_t used = 0;
    while (j < sorted.size() && used + sorted[j].tb_words <= budget) used += sorted[j++].tb_words;
    // group the slice [i, j) by kernel shape, stable (keeps the cost order)
    Wave w;
    w.tb_words = used;
    std::vector<PairPlan> slice(sorted.begin() + i, sorted.begin() + j);
    std::stable_sort(slice.begin(), slice.end(), [](const PairPlan &a, const PairPlan &b) {
      if (a.family != b.family) return a.family < b.family;
      if (a.R != b.R) return a.R > b.R;
      return a.warps > b.warps;
    });
    const uint32_t wave_begin = (uint32_t)P->order.size();
    uint64_t off = 0;
    size_t g0 = 0;
    for (size_t t = 0; t < slice.size(); ++t) {
      const PairPlan &x = slice[t];
      TbLayout &L = P->tbl[x.pair];
      L.off = off;
      L.family = x.family;
      L.R = x.R;
      L.warps = x.warps;
      L.valid = sp.traceback ? 1 : 0;
      off += x.tb_words;
      P->order.push_back(x.pair);
      const bool last = (t + 1 == slice.size());
      if (last || slice[t + 1].family != x.family || slice[t + 1].R != x.R ||
          slice[t + 1].warps != x.warps) {
        Group g;
        g.family = x.family;
        g.R = x.R;
        g.warps = x.warps;
        g.begin = wave_begin + (uint32_t)g0;
        g.end = wave_begin + (uint32_t)(t + 1);
        w.groups.push_back(g);
        g0 = t + 1;
      }
    }
    w.walk_begin = wave_begin;
    w.walk_end = (uint32_t)P->order.size();
    P->waves.push_back(w);
    i = j;
  }
  return true;
}

}  // namespace filtr
