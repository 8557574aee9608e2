// plan_pair.h -- per-pair planning rules shared by the host planner (plan.cpp)
// and the device planner (k_plan.cu): cell counts, tile strips, traceback words,
// cost buckets and the choice of tiled kernel shape.  Both planners call these
// same functions, so they give every pair the same shape.
#pragma once

#include "filtr_internal.h"

namespace filtr {

// Tiled kernel shapes (int32 R = 32, 24, 16, 8; int16x2 R = 32, 30, ..., 10,
// 8), then X-drop.
enum : int { SHAPE_TILED = 17, SHAPE_XDROP = 17, SHAPE_KEYS = 18 };
struct ShapeCost {
  int R, fill;        // rows per lane; fill steps per strip (staircase)
  float per_row;      // cost of one row (int32) or one packed register pair of rows / 2
  float per_step;     // per-step overhead of a lane
  bool packed;
};

// ceil(M / 32R) for even R from 8 to 32: tile heights are multiples of 64
// rows, and ceil(ceil(M / 64) / (R / 2)) = ceil(M / 32R), so one shift and a
// division by a small constant give every height.
FILTR_HD uint32_t strips_s64(uint32_t s64, int d) {  // ceil(s64 / d), d = R / 2
  switch (d) {
    case 4: return (s64 + 3u) >> 2;
    case 5: return (s64 + 4u) / 5u;
    case 6: return (s64 + 5u) / 6u;
    case 7: return (s64 + 6u) / 7u;
    case 8: return (s64 + 7u) >> 3;
    case 9: return (s64 + 8u) / 9u;
    case 10: return (s64 + 9u) / 10u;
    case 11: return (s64 + 10u) / 11u;
    case 12: return (s64 + 11u) / 12u;
    case 13: return (s64 + 12u) / 13u;
    case 14: return (s64 + 13u) / 14u;
    case 15: return (s64 + 14u) / 15u;
    default: return (s64 + 15u) >> 4;
  }
}
FILTR_HD uint64_t strips_of(uint32_t M, int R) {
  if (R % 2 != 0 || R < 8 || R > 32) return ((uint64_t)M + 32u * R - 1) / (32u * R);
  return strips_s64((uint32_t)(((uint64_t)M + 63u) >> 6), R / 2);
}

// Traceback words of one pair in the int32 tile of R rows per lane.
FILTR_HD uint64_t full_tb_words(uint32_t M, uint32_t N, int R, const ScoreParams &sp) {
  const int64_t HS = 32 * R;
  if (!sp.use_band) return strips_of(M, R) * (uint64_t)strip_tb_words(1, N, R);
  int64_t lo, hi;
  band_limits(M, N, sp.band, sp.band_literal != 0, &lo, &hi);
  uint64_t w = 0;
  const int64_t ns = ((int64_t)M + HS - 1) / HS;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t jl, jh;
    strip_cols(s * HS, HS, M, N, true, lo, hi, &jl, &jh);
    if (jl > jh) break;
    w += (uint64_t)strip_tb_words(jl, jh, R);
  }
  return w;
}

// Cell count of one pair under a static band (or the full matrix): the sum over
// diagonals d in [lo, hi] of the cells of diagonal d inside the matrix,
// f(d) = min(M, N - d) - max(0, -d) for 1-M <= d <= N-1.  f is linear between
// its kinks at d = 0 and d = N - M, so each piece is an arithmetic sum.
FILTR_HD uint64_t band_cells(uint32_t M, uint32_t N, const ScoreParams &sp) {
  if (!sp.use_band) return (uint64_t)M * N;
  int64_t lo, hi;
  band_limits(M, N, sp.band, sp.band_literal != 0, &lo, &hi);
  const int64_t Mi = M, Ni = N;
  const int64_t A = lo > 1 - Mi ? lo : 1 - Mi, B = hi < Ni - 1 ? hi : Ni - 1;
  if (A > B) return 0;
  const int64_t k1 = Ni - Mi < 0 ? Ni - Mi : 0, k2 = Ni - Mi > 0 ? Ni - Mi : 0;
  auto clamp = [&](int64_t k) {
    const int64_t v = k > A - 1 ? k : A - 1;
    return v < B ? v : B;
  };
  auto f = [&](int64_t d) {
    const int64_t a = Mi < Ni - d ? Mi : Ni - d;
    return a - (d < 0 ? -d : 0);
  };
  const int64_t cut[4] = {A - 1, clamp(k1), clamp(k2), B};
  uint64_t c = 0;
  for (int s = 0; s < 3; ++s) {
    const int64_t a = cut[s] + 1, b = cut[s + 1];
    if (b >= a) c += (uint64_t)((f(a) + f(b)) * (b - a + 1) / 2);
  }
  return c;
}

// Half-octave cost bucket, 2 * floor(log2(cost)) + the next bit, reversed so
// that bucket 0 holds the most expensive pairs.
FILTR_HD int cost_bucket_desc(uint64_t cost) {
  if (cost < 2) return 63;
#ifdef __CUDA_ARCH__
  const int lg = 63 - __clzll((long long)cost);
#else
  const int lg = 63 - __builtin_clzll(cost);
#endif
  const int b = 2 * lg + (int)((cost >> (lg - 1)) & 1);
  return 63 - (b < 63 ? b : 63);
}

// The shape costs in the form the per-pair choice reads them.
struct ShapeTable {
  double coef[SHAPE_TILED];  // per_row x R + per_step
  double fill[SHAPE_TILED];
  int R[SHAPE_TILED];
  int packed[SHAPE_TILED];
  int elig[SHAPE_TILED];     // shapes the recurrence kind allows, in table order
  int n_elig, n_elig_packed;
};

inline ShapeTable make_shape_table(const ShapeCost *costs, const ScoreParams &sp) {
  ShapeTable t{};
  const bool pack_ok = !sp.use_band && !sp.use_xdrop && sp.precision != FILTR_PREC_I32;
  for (int k = 0; k < SHAPE_TILED; ++k) {
    t.coef[k] = (double)costs[k].per_row * costs[k].R + costs[k].per_step;
    t.fill[k] = (double)costs[k].fill;
    t.R[k] = costs[k].R;
    t.packed[k] = costs[k].packed ? 1 : 0;
    if (costs[k].packed && !pack_ok) continue;
    t.elig[t.n_elig++] = k;
    t.n_elig_packed += costs[k].packed ? 1 : 0;
  }
  return t;
}

// The cheapest allowed tiled shape for an M x N pair: strips x (N + fill) x
// cost per warp step; the int16x2 tile only where the pair's static score
// bound fits 15 bits, and then always under FILTR_PREC_I16X2.  The minimum is
// taken without branches (the winner changes from pair to pair); ties go to the
// earlier shape of the table.
FILTR_HD int choose_shape_p(const ShapeTable &t, bool packable, bool only_packed, uint32_t M,
                            uint32_t N) {
  const uint32_t s64 = (uint32_t)(((uint64_t)M + 63u) >> 6);
  const double Nd = (double)N;
  int best = t.elig[0];
  double bc = 1e300;
  for (int i = 0; i < t.n_elig; ++i) {
    const int k = t.elig[i];
    const bool skip = t.packed[k] ? !packable : only_packed;
    double c = (double)strips_s64(s64, t.R[k] / 2) * (Nd + t.fill[k]) * t.coef[k];
    c = skip ? 1e300 : c;
    const bool lt = c < bc;
    best = lt ? k : best;
    bc = lt ? c : bc;
  }
  return best;
}
FILTR_HD int choose_shape(const ShapeTable &t, const ScoreParams &sp, uint32_t M, uint32_t N) {
  const bool packable =
      t.n_elig_packed > 0 && pack_bias(sp.mode, sp.o, sp.e, sp.smin, sp.smax, M, N) >= 0;
  return choose_shape_p(t, packable, packable && sp.precision == FILTR_PREC_I16X2, M, N);
}

// Traceback words of an M x N pair in shape k.
FILTR_HD uint64_t shape_tb_words(const ShapeTable &t, int k, uint32_t M, uint32_t N,
                                 const ScoreParams &sp) {
  return t.packed[k] ? strips_of(M, t.R[k]) * pack_strip_tb_words(1, N, t.R[k])
                     : full_tb_words(M, N, t.R[k], sp);
}

}  // namespace filtr
