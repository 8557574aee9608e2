// plan.h -- host planner for one batched call: kernel shape per pair, length /
// cost ordering, traceback waves and the device workspace layout.
#pragma once

#include <stdint.h>

#include <vector>

#include "filtr_internal.h"

namespace filtr {

struct Group {          // pairs of one wave that share one kernel instance
  uint8_t family, R, warps;
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
};

// Tiled kernel shapes (int32 and int16x2, R = 32, 24, 16, 8), then X-drop.
enum : int { SHAPE_TILED = 8, SHAPE_XDROP = 8, SHAPE_KEYS = 9 };
struct ShapeCost {
  int R, fill;        // rows per lane; fill steps per strip (staircase)
  float per_row;      // cost of one row (int32) or one packed register pair of rows / 2
  float per_step;     // per-step overhead of a lane
  bool packed;
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
// Traceback words of one pair in the tiled kernel.
uint64_t full_tb_words(uint32_t M, uint32_t N, int R, const ScoreParams &sp);
// Cell count of one pair under a static band (or the full matrix).
uint64_t band_cells(uint32_t M, uint32_t N, const ScoreParams &sp);

// Returns false (and sets the error message) if a single pair cannot fit.
bool make_plan(const PlanInput &in, Plan *out);

}  // namespace filtr
