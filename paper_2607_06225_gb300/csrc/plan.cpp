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
    {8, 31, 16.0f, 30.0f, false},  {32, 63, 12.0f, 40.0f, true},  {24, 63, 12.0f, 40.0f, true},
    {16, 63, 12.0f, 40.0f, true},  {8, 63, 12.0f, 40.0f, true}};

double shape_cost(const ShapeCost &c, uint32_t M, uint32_t N) {
  const uint64_t hs = 32u * c.R;
  const uint64_t strips = (M + hs - 1) / hs;
  return (double)strips * (double)(N + c.fill) * ((double)c.per_row * c.R + c.per_step);
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

uint64_t full_tb_words(uint32_t M, uint32_t N, int R, const ScoreParams &sp) {
  const int64_t HS = 32 * R;
  const bool band = sp.use_band != 0;
  if (!band) return (uint64_t)((M + HS - 1) / HS) * (uint64_t)strip_tb_words(1, N, R);
  int64_t lo = -(int64_t)M - 1, hi = (int64_t)N + 1;
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

// half-octave buckets: 2 * floor(log2(cost)) + the next bit
static int cost_bucket(uint64_t cost) {
  if (cost < 2) return 0;
  const int lg = 63 - __builtin_clzll(cost);
  const int b = 2 * lg + (int)((cost >> (lg - 1)) & 1);
  return b < 63 ? b : 63;
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

  // per pair: kernel shape key, cost bucket, traceback words (flat arrays)
  // shape keys: 0..3 the int32 tiled kernel with R = 32, 24, 16, 8; 4..7 the
  // int16x2 tiled kernel with R = 32, 24, 16, 8; 8 the X-drop kernel
  const ShapeCost *costs = in.shape_cost ? in.shape_cost : kDefaultShapeCost;
  const bool pack_ok = !sp.use_band && !sp.use_xdrop && sp.precision != FILTR_PREC_I32;
  std::vector<uint8_t> bucket(n), shape(n);
  std::vector<uint64_t> words(n);
  std::vector<uint32_t> cnt(64, 0);
  const int xw = in.xdrop_warps > 0
                     ? in.xdrop_warps
                     : (sp.use_xdrop ? xdrop_first_width(sp, n, in.q_len, in.r_len, in.xdrop_slots) : 1);
  P->xdrop_w0 = xw;
  uint32_t live = 0;
  for (uint32_t p = 0; p < n; ++p) {
    const uint32_t M = in.q_len[p], N = in.r_len[p];
    if (N > P->max_n) P->max_n = N;
    if (M > P->max_m) P->max_m = M;
    P->cigar_upper += (uint64_t)M + N;
    if (sp.traceback) {
      P->stage_off[p] = P->stage_words;
      P->stage_words += (uint64_t)M + N + 1;
    }
    // an empty side leaves no cell to evaluate, except under X-drop, where the
    // gap cells of row 0 / column 0 are themselves subject to the prune test
    if ((M == 0 && N == 0) || ((M == 0 || N == 0) && !sp.use_xdrop)) {
      P->trivial.push_back(p);
      shape[p] = 255;
      continue;
    }
    const uint64_t cost = band_cells(M, N, sp);
    P->cells_estimate += cost;
    uint64_t w = 0;
    if (sp.use_xdrop) {
      shape[p] = SHAPE_XDROP;
      if (sp.traceback) w = xd_tb_words(M, N, xw, in.xdrop_slots);
    } else {
      // cheapest eligible shape; FILTR_PREC_I16X2 takes the packed kernel
      // whenever the pair's score range fits it
      const bool packable =
          pack_ok && pack_bias(sp.mode, sp.o, sp.e, sp.smin, sp.smax, M, N) >= 0;
      int best = -1;
      double bc = 0;
      for (int k = 0; k < SHAPE_TILED; ++k) {
        if (costs[k].packed && !packable) continue;
        if (sp.use_band && costs[k].packed) continue;
        if (packable && sp.precision == FILTR_PREC_I16X2 && !costs[k].packed) continue;
        const double c = shape_cost(costs[k], M, N);
        if (best < 0 || c < bc) {
          best = k;
          bc = c;
        }
      }
      shape[p] = (uint8_t)best;
      const ShapeCost &sc = costs[best];
      if (sp.traceback)
        w = sc.packed ? (uint64_t)((M + 32u * sc.R - 1) / (32u * sc.R)) * pack_strip_tb_words(1, N, sc.R)
                      : full_tb_words(M, N, sc.R, sp);
    }
    if (sp.traceback && w > in.tb_budget_words) {
      set_error("pair %u needs %llu traceback bytes, more than the workspace allows", p,
                (unsigned long long)(w * 4));
      return false;
    }
    words[p] = w;
    bucket[p] = (uint8_t)(63 - cost_bucket(cost));
    cnt[bucket[p]]++;
    ++live;
  }

  // counting sort of pair ids, most expensive bucket first
  std::vector<uint32_t> start(64, 0);
  for (int b = 1; b < 64; ++b) start[b] = start[b - 1] + cnt[b - 1];
  std::vector<uint32_t> sorted(live);
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
