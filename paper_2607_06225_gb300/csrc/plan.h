// plan.h -- host planner for one batched call: kernel shape per pair, length /
// cost ordering, traceback waves and the device workspace layout.
#pragma once

#include <stdint.h>

#include <vector>

#include "filtr_internal.h"
#include "plan_pair.h"

namespace filtr {

struct Group {          // pairs of one wave that share one kernel instance
  uint8_t family, R, warps;
  int8_t shape = -1;    // tiled shape index (device plan), -1 otherwise
  uint32_t begin, end;  // slice of Plan::order
};

struct Wave {
  std::vector<Group> groups;
  uint32_t walk_begin, walk_end;  // slice of Plan::order whose traceback is walked after this wave
  uint64_t tb_words;              // traceback words used by this wave
};

struct Plan {
  std::vector<uint32_t> order;    // pair ids, grouped per wave and group, cost-descending inside a group
  std::vector<TbLayout> tbl;      // per pair id
  std::vector<uint64_t> stage_off;  // per pair id (CIGAR staging, in words)
  std::vector<Wave> waves;
  std::vector<uint32_t> trivial;  // pairs with an empty sequence
  uint64_t stage_words = 0;
  uint64_t max_n = 0, max_m = 0;
  uint64_t cigar_upper = 0;       // sum over pairs of M + N: no CIGAR can be longer
  int xdrop_w0 = 1;               // group width X-drop / Z-drop pairs first run at
  uint64_t cells_estimate = 0;
  uint64_t cells_packed = 0;  // of which in pairs given an int16x2 shape
  // per-pair scratch of make_plan, kept with the plan so that a context that
  // plans batch after batch reuses its pages
  std::vector<uint8_t> s_bucket, s_shape;
  std::vector<uint64_t> s_words;
  std::vector<uint32_t> s_sorted;
};

extern const ShapeCost kDefaultShapeCost[SHAPE_TILED];
double shape_cost(const ShapeCost &c, uint32_t M, uint32_t N);

struct PlanInput {
  const ScoreParams *sp;
  uint32_t n;
  const uint32_t *q_len, *r_len;  // host copies
  uint64_t tb_budget_words;       // traceback words one wave may use
  int xdrop_slots;                // slots per lane of the X-drop kernel
  int xdrop_warps;                // first window width of X-drop pairs (warps), 0: estimated
  const ShapeCost *shape_cost = nullptr;  // nullptr: kDefaultShapeCost
};

// First group width (warps) for X-drop / Z-drop pairs, from the expected width
// of their live region (see plan.cpp).
int xdrop_first_width(const ScoreParams &sp, uint32_t n, const uint32_t *q_len,
                      const uint32_t *r_len, int slots);

// Rows per lane of the tiled kernel for an M x N pair.
int full_rows_per_lane(uint32_t M, uint32_t N);

// Returns false (and sets the error message) if a single pair cannot fit.
bool make_plan(const PlanInput &in, Plan *out);

// ---- the same plan built on the device (tiled batches in one wave) ----
//
// Three launches over the pairs: classify (shape and cost bucket of each pair,
// a block histogram of the keys, block sums of the CIGAR staging words and
// batch totals), scan (key histogram and block sums to starting offsets), and
// place (pair ids scattered into shape-major, cost-descending order with
// warp-aggregated atomics; disjoint traceback offsets; staging offsets in pair
// order).  Pairs with an empty side take key KEY_TRIVIAL, after every shape.
// Shapes and buckets are those make_plan gives; the order inside one (shape,
// bucket) cell and the placement of traceback areas depend on atomics, which
// changes no result.
enum : int { KEY_TRIVIAL = SHAPE_TILED, PLAN_KEYS = (SHAPE_TILED + 1) * 64 };

struct DevPlanSummary {
  uint32_t count[SHAPE_TILED + 1];  // pairs per tiled shape, then empty pairs
  uint32_t max_m, max_n;
  uint32_t pad;
  unsigned long long tb_words;      // traceback words of all pairs
  unsigned long long cells;         // cells of the non-empty pairs
  unsigned long long stage_words;   // sum of M + N + 1 (traceback on)
  unsigned long long cigar_upper;   // sum of M + N
  unsigned long long cells_packed;  // cells of the pairs given an int16x2 shape
};

// Zeroed before each call.  The host reads back bad[] and sum with one copy.
struct DevPlanState {
  uint32_t bad[64];                 // residue validation count in bad[0]
  DevPlanSummary sum;
  uint32_t hist[PLAN_KEYS];
  uint32_t cursor[PLAN_KEYS];
  unsigned long long tb_cursor;
};

struct DevPlanArgs {
  const uint32_t *q_len, *r_len;
  uint32_t n;
  ScoreParams sp;
  ShapeTable tab;
  DevPlanState *state;
  uint16_t *key;        // per pair: shape * 64 + bucket
  uint64_t *words;      // per pair: traceback words
  uint64_t *blk;        // per block of DEV_PLAN_BLOCK pairs: staging words, then base
  uint32_t *order;      // out: pair ids
  TbLayout *tbl;        // out: per pair
  uint64_t *stage_off;  // out: per pair (traceback on)
  const GraphDesc *gd = nullptr;  // captured pipeline: n (at most the n above) and lengths from here
};
constexpr int DEV_PLAN_BLOCK = 256;
cudaError_t launch_plan(const DevPlanArgs &a, cudaStream_t st);

#ifdef __CUDACC__
// What one tiled launch works on.  The batched call's instances (GR = false)
// read their by-value arguments, which live in the parameter bank and cost no
// register.  A captured pipeline's instances (GR = true) take the batch and
// outputs from the graph descriptor and their slice of the order from the
// device plan, read per pair (volatile: never hoisted into registers that
// live across the persistent loop).
template <bool GR>
__device__ __forceinline__ uint32_t launch_n(const FullArgs &a) {
  if constexpr (GR) {
    const volatile DevPlanSummary *s = a.gsum;
    return s->count[a.gshape];
  } else {
    return a.n_order;
  }
}
template <bool GR>
__device__ __forceinline__ const uint32_t *launch_order(const FullArgs &a) {
  if constexpr (GR) {
    const volatile DevPlanSummary *s = a.gsum;
    uint32_t begin = 0;
    for (int k = 0; k < a.gshape; ++k) begin += s->count[k];
    return a.order + begin;
  } else {
    return a.order;
  }
}
template <bool GR>
__device__ __forceinline__ BatchDev launch_batch(const FullArgs &a) {
  if constexpr (GR) {
    const volatile GraphDesc *g = a.gd;
    BatchDev b;
    b.q_seq = g->b.q_seq;
    b.r_seq = g->b.r_seq;
    b.q_off = g->b.q_off;
    b.r_off = g->b.r_off;
    b.q_len = g->b.q_len;
    b.r_len = g->b.r_len;
    return b;
  } else {
    return a.b;
  }
}
template <bool GR>
__device__ __forceinline__ filtr_result *launch_out(const FullArgs &a) {
  if constexpr (GR) {
    const volatile GraphDesc *g = a.gd;
    return g->out;
  } else {
    return a.out;
  }
}
// Nothing to do (captured pipeline): the pipeline was aborted, or the
// persistent grid (sized for the whole device) has more blocks than this
// shape has pairs.
template <bool GR>
__device__ __forceinline__ bool launch_idle(const FullArgs &a) {
  if constexpr (GR) {
    return a.gd->abort != 0 || (uint64_t)blockIdx.x * FULL_WARPS >= launch_n<GR>(a);
  } else {
    return false;
  }
}
#endif

}  // namespace filtr
