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

#include "k_xdrop_layout.h"

namespace filtr {

// Kernel shapes of the unbanded / banded tiled path and their cost model:
// a shape costs strips x (N + fill) steps x (per_row x rows + per_step) per
// lane, with the coefficients in issue-slot units (defaults from the measured
// instruction mix; filtr_autotune replaces them with timed values).
const ShapeCost kDefaultShapeCost[SHAPE_TILED] = {
    {32, 31, 16.0f, 30.0f, false}, {24, 31, 16.0f, 30.0f, false}, {16, 31, 16.0f, 30.0f, false},
    {8, 31, 16.0f, 30.0f, false},  {32, 63, 12.0f, 40.0f, true},  {30, 63, 12.0f, 40.0f, true},
    {28, 63, 12.0f, 40.0f, true},  {26, 63, 12.0f, 40.0f, true},  {24, 63, 12.0f, 40.0f, true},
    {22, 63, 12.0f, 40.0f, true},  {20, 63, 12.0f, 40.0f, true},  {18, 63, 12.0f, 40.0f, true},
    {16, 63, 12.0f, 40.0f, true},  {14, 63, 12.0f, 40.0f, true},  {12, 63, 12.0f, 40.0f, true},
    {10, 63, 12.0f, 40.0f, true},  {8, 63, 12.0f, 40.0f, true}};

double shape_cost(const ShapeCost &c, uint32_t M, uint32_t N) {
  return (double)strips_of(M, c.R) * (double)(N + c.fill) * ((double)c.per_row * c.R + c.per_step);
}

// Rows per lane: the tile height 32R whose padded work, strips x (N + 31 steps)
// x (R + 2) (two cell-equivalents of per-step overhead), is smallest.
int full_rows_per_lane(uint32_t M, uint32_t N) {
  static const int Rs[4] = {32, 24, 16, 8};
  int best = 8;
  uint64_t best_cost = ~0ull;
  for (int R : Rs) {
    const uint64_t strips = (M + 32u * R - 1) / (32u * R);
    const uint64_t cost = strips * ((uint64_t)N + 31) * (uint64_t)(R + 2);
    if (cost < best_cost) {
      best_cost = cost;
      best = R;
    }
  }
  return best;
}

// X-drop / Z-drop live region: a cell delta places off the best cell along an
// antidiagonal sits 2*delta diagonals away, which takes gaps costing about
// o + 2*delta*e.  X-drop keeps it while that stays within X, so about
// (X - o) / e cells live; Z-drop adds one per diagonal of distance to the
// threshold, so about (Z - o) / (e - 1) (no bound when e <= 1).  The band and
// the matrix cap both.  The first group is the narrowest whose window holds the
// estimate; pairs that outgrow it are rerun wider, so a low estimate costs a
// partial pass, a high one a wider (slower) sweep.
int xdrop_first_width(const ScoreParams &sp, uint32_t n, const uint32_t *q_len,
                      const uint32_t *r_len, int slots) {
  const double X = (double)sp.xdrop, o = (double)sp.o, e = (double)sp.e;
  double est = 1e18;
  if (sp.xdrop < FILTR_XDROP_INF) {
    if (!sp.zdrop && e > 0) est = std::max(1.0, (X - o) / e);
    if (sp.zdrop && e > 1) est = std::max(1.0, (X - o) / (e - 1));
  }
  double cap = 0;
  for (uint32_t p = 0; p < n; ++p) {
    double c = (double)std::min(q_len[p], r_len[p]) + 1;
    if (sp.use_band) {
      int64_t lo, hi;
      band_limits(q_len[p], r_len[p], sp.band, sp.band_literal, &lo, &hi);
      c = std::min(c, (double)(hi - lo) / 2 + 1);
    }
    cap = std::max(cap, c);
  }
  est = std::min(est, cap);
  for (int W : {1, 2, 4, 8, 16}) if ((double)W * 32 * slots >= est) return W;
  return 32;
}

bool make_plan(const PlanInput &in, Plan *P) {
  const ScoreParams &sp = *in.sp;
  const uint32_t n = in.n;
  P->order.clear();
  P->order.reserve(n);
  P->tbl.assign(n, TbLayout{});
  P->stage_off.assign(n, 0);
  P->waves.clear();
  P->trivial.clear();
  P->stage_words = 0;
  P->max_n = P->max_m = 0;
  P->cigar_upper = 0;
  P->cells_estimate = 0;
  P->cells_packed = 0;

  // per pair: kernel shape key, cost bucket, traceback words (flat arrays)
  // shape keys: 0..3 the int32 tiled kernel with R = 32, 24, 16, 8; 4..7 the
  // int16x2 tiled kernel with R = 32, 24, 16, 8; 8 the X-drop kernel
  const ShapeCost *costs = in.shape_cost ? in.shape_cost : kDefaultShapeCost;
  const ShapeTable tab = make_shape_table(costs, sp);
  P->s_bucket.resize(n);
  P->s_shape.resize(n);
  P->s_words.resize(n);
  uint8_t *bucket = P->s_bucket.data(), *shape = P->s_shape.data();
  uint64_t *words = P->s_words.data();
  uint32_t cnt[64] = {};
  const int xw = in.xdrop_warps > 0
                     ? in.xdrop_warps
                     : (sp.use_xdrop ? xdrop_first_width(sp, n, in.q_len, in.r_len, in.xdrop_slots) : 1);
  P->xdrop_w0 = xw;
  uint32_t live = 0;
  // running totals in locals: the byte stores below may alias *P
  uint64_t max_n = 0, max_m = 0, cigar_upper = 0, stage_words = 0, cells = 0, cells_packed = 0;
  uint64_t *stage_off = P->stage_off.data();
  for (uint32_t p = 0; p < n; ++p) {
    const uint32_t M = in.q_len[p], N = in.r_len[p];
    max_n = N > max_n ? N : max_n;
    max_m = M > max_m ? M : max_m;
    cigar_upper += (uint64_t)M + N;
    if (sp.traceback) {
      stage_off[p] = stage_words;
      stage_words += (uint64_t)M + N + 1;
    }
    // an empty side leaves no cell to evaluate, except under X-drop, where the
    // gap cells of row 0 / column 0 are themselves subject to the prune test
    if ((M == 0 && N == 0) || ((M == 0 || N == 0) && !sp.use_xdrop)) {
      P->trivial.push_back(p);
      shape[p] = 255;
      continue;
    }
    const uint64_t cost = band_cells(M, N, sp);
    cells += cost;
    uint64_t w = 0;
    if (sp.use_xdrop) {
      shape[p] = SHAPE_XDROP;
      if (sp.traceback) w = xd_tb_words(M, N, xw, in.xdrop_slots);
    } else {
      const int k = choose_shape(tab, sp, M, N);
      shape[p] = (uint8_t)k;
      if (tab.packed[k]) cells_packed += cost;
      if (sp.traceback) w = shape_tb_words(tab, k, M, N, sp);
    }
    if (sp.traceback && w > in.tb_budget_words) {
      set_error("pair %u needs %llu traceback bytes, more than the workspace allows", p,
                (unsigned long long)(w * 4));
      return false;
    }
    words[p] = w;
    bucket[p] = (uint8_t)cost_bucket_desc(cost);
    cnt[bucket[p]]++;
    ++live;
  }
  P->max_n = max_n;
  P->max_m = max_m;
  P->cigar_upper = cigar_upper;
  P->stage_words = stage_words;
  P->cells_estimate = cells;
  P->cells_packed = cells_packed;

  // counting sort of pair ids, most expensive bucket first
  uint32_t start[64] = {};
  for (int b = 1; b < 64; ++b) start[b] = start[b - 1] + cnt[b - 1];
  P->s_sorted.resize(live);
  std::vector<uint32_t> &sorted = P->s_sorted;
  for (uint32_t p = 0; p < n; ++p)
    if (shape[p] != 255) sorted[start[bucket[p]]++] = p;

  // waves: cut the cost order where the traceback budget is used up, then
  // group each wave by kernel shape (stable counting sort over the keys)
  const uint64_t budget = sp.traceback ? in.tb_budget_words : ~0ull;
  size_t i = 0;
  while (i < sorted.size()) {
    size_t j = i;
    uint64_t used = 0;
    uint32_t kc[SHAPE_KEYS] = {};
    while (j < sorted.size() && used + words[sorted[j]] <= budget) {
      used += words[sorted[j]];
      kc[shape[sorted[j]]]++;
      ++j;
    }
    Wave w;
    w.tb_words = used;
    const uint32_t wave_begin = (uint32_t)P->order.size();
    uint32_t ks[SHAPE_KEYS], kpos[SHAPE_KEYS];
    ks[0] = wave_begin;
    for (int k = 1; k < SHAPE_KEYS; ++k) ks[k] = ks[k - 1] + kc[k - 1];
    P->order.resize(wave_begin + (j - i));
    for (int k = 0; k < SHAPE_KEYS; ++k) kpos[k] = ks[k];
    for (size_t t = i; t < j; ++t) P->order[kpos[shape[sorted[t]]]++] = sorted[t];
    // traceback offsets in wave order, per-pair layout, groups
    uint64_t off = 0;
    for (int k = 0; k < SHAPE_KEYS; ++k) {
      if (!kc[k]) continue;
      Group g;
      if (k == SHAPE_XDROP) {
        g.family = FAM_XDROP;
        g.R = (uint8_t)in.xdrop_slots;
        g.warps = (uint8_t)xw;
      } else {
        g.family = costs[k].packed ? FAM_PACK : FAM_FULL;
        g.R = (uint8_t)costs[k].R;
        g.warps = 1;
      }
      g.begin = ks[k];
      g.end = ks[k] + kc[k];
      for (uint32_t t = g.begin; t < g.end; ++t) {
        const uint32_t p = P->order[t];
        TbLayout &L = P->tbl[p];
        L.off = off;
        L.family = g.family;
        L.R = g.R;
        L.warps = g.warps;
        L.valid = sp.traceback ? 1 : 0;
        off += words[p];
      }
      w.groups.push_back(g);
    }
    w.walk_begin = wave_begin;
    w.walk_end = (uint32_t)P->order.size();
    P->waves.push_back(w);
    i = j;
  }
  return true;
}

}  // namespace filtr
