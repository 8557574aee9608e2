// filtr_ctx.h -- the context object behind the opaque filtr_ctx handle.
#pragma once

#include <algorithm>
#include <cstdlib>
#include <map>
#include <tuple>

#include "filtr_internal.h"
#include "plan.h"

namespace filtr {

struct Ctx {
  int device = 0;
  int sms = 0;
  char *ws = nullptr;         // device workspace (plan, staging, traceback)
  size_t ws_bytes = 0;
  void *h_stage = nullptr;    // pinned host staging
  size_t h_stage_bytes = 0;
  void *d_io = nullptr;       // device copies for the host-buffer entry point
  char *d_small = nullptr;    // 4 KiB of device memory for per-call scalars
  size_t d_io_bytes = 0;
  cudaStream_t own_stream = nullptr;
  // side streams and fork / join events for tiled shapes launched concurrently
  std::vector<cudaStream_t> side;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  bool ensure_side(int n);
  std::map<std::tuple<int, int, int, int, int, int>, int> occ_cache;
  uint64_t last_cells_estimate = 0;
  uint64_t last_cells_packed = 0;
  uint32_t last_xd16 = 0, last_xd16_rerun = 0;
  int xd16_mode = 0;  // packed antidiagonal sweep: 0 when eligible, 1 never, 2 without moving the base
  uint32_t last_pairs_packed = 0;
  double last_host_wait_ms = 0, last_host_plan_ms = 0;
  Plan plan;                       // the last call's plan; its buffers are reused
  int dev_plan_mode = 0;           // 0: device planner by batch size, 1: never, 2: always
  int search_ring = 0;             // search score pass: shared-memory ring entries, 0 default
  bool last_dev_plan = false;      // the last call was planned on the device
  std::vector<uint32_t> h_ql, h_rl;  // the last call's lengths (host copies)
  int last_waves = 0;
  uint32_t last_launches = 0;
  int xdrop_warps0 = 0;       // first window width (warps) of X-drop pairs, 0: estimated
  int ckpt_interval = 0;      // > 0: filtr_align_long always checkpoints X-drop tracebacks
  bool ckpt_recompute = false;  // checkpointed traceback: recompute segments, no single pass
  // ordering of successive calls: the next call waits for this event, so the
  // workspace and the pinned staging are never reused while still in flight
  cudaEvent_t done_ev = nullptr;
  // optional per-phase timing
  bool timing = false;
  enum Phase { PH_VALIDATE = 0, PH_FORWARD = 1, PH_WALK = 2, PH_PLACE = 3 };
  struct Span {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Span> spans;

  // measured shape costs (filtr_autotune), per recurrence kind
  // the antidiagonal sweep's tuned choice (filtr_autotune with X-drop / Z-drop
  // parameters): cell width and first group width, per recurrence kind
  struct SweepChoice {
    int packed, warps;
  };
  using SweepKey = std::tuple<int, int, int, int, int, int>;  // mode, alphabet, traceback, band, zdrop, running
  std::map<SweepKey, SweepChoice> sweep_tuned;
  static SweepKey sweep_key(const ScoreParams &sp) {
    return SweepKey(sp.mode, sp.alphabet, sp.traceback, sp.use_band, sp.zdrop, sp.xrun);
  }
  const SweepChoice *sweep_choice(const ScoreParams &sp) const {
    auto it = sweep_tuned.find(sweep_key(sp));
    return it == sweep_tuned.end() ? nullptr : &it->second;
  }
  using TuneKey = std::tuple<int, int, int, int, int>;  // mode, affine, traceback, alphabet, band
  std::map<TuneKey, std::vector<ShapeCost>> tuned;
  static TuneKey tune_key(const ScoreParams &sp) {
    return TuneKey(sp.mode, sp.affine, sp.traceback, sp.alphabet, sp.use_band);
  }
  const ShapeCost *tuned_costs(const ScoreParams &sp) const {
    auto it = tuned.find(tune_key(sp));
    return it == tuned.end() ? nullptr : it->second.data();
  }

  int full_blocks_per_sm(int R, const ScoreParams &sp);
  int pack_blocks_per_sm(int R, const ScoreParams &sp);
  int graph_blocks_per_sm(int R, bool packed, const ScoreParams &sp);  // filtr_graph instances
  bool ensure_host(size_t bytes);
  cudaEvent_t next_event();
  // open / close a timed span on stream st (no-ops when timing is off)
  void span_begin(int phase, cudaStream_t st);
  void span_end(cudaStream_t st);
};

filtr_status to_score_params(const filtr_params *p, ScoreParams *sp);
// prevalidated: the caller checked every residue code on the host and passes
// host_ql / host_rl, so the call needs no host synchronisation up front.
filtr_status align_batch_impl(Ctx *ctx, const filtr_params *params, uint32_t n, const BatchDev &b,
                              filtr_result *out, uint32_t *cigar, uint64_t cap, cudaStream_t st,
                              bool plain, const uint32_t *host_ql, const uint32_t *host_rl,
                              bool prevalidated);
filtr_status ctx_new(int device, size_t workspace_bytes, Ctx **out);
// one long full-matrix / banded pair across the grid, not waited for
filtr_status long_pair_async(Ctx *c, const ScoreParams &sp, const filtr_params *params,
                             const uint8_t *q, uint32_t M, const uint8_t *r, uint32_t N,
                             filtr_result *out, uint32_t *cigar, uint64_t cap, cudaStream_t st);
void ctx_delete(Ctx *c);

}  // namespace filtr
