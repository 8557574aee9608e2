// api.cu -- the C ABI (include/filtr.h): contexts, parameter checks, the
// batched call (plan, wave launches, traceback walk, CIGAR placement), its
// host-buffer and per-pair-launch variants, packing and the throughput probe.
#include <chrono>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/filtr_testing.h"
#include "filtr_ctx.h"
#include "k_xdrop_layout.h"
#include "plan.h"

namespace filtr {

static thread_local std::string g_err = "no error";

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

filtr_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return FILTR_ERR_CUDA;
}

filtr_status to_score_params(const filtr_params *p, ScoreParams *sp) {
  if (!p) {
    set_error("params is NULL");
    return FILTR_ERR_INVALID;
  }
  if (p->mode != FILTR_GLOBAL && p->mode != FILTR_LOCAL) {
    set_error("mode must be FILTR_GLOBAL or FILTR_LOCAL");
    return FILTR_ERR_INVALID;
  }
  if (p->alphabet != FILTR_ALPHA_DNA && p->alphabet != FILTR_ALPHA_PROTEIN) {
    set_error("alphabet must be 4 (DNA) or 20 (protein)");
    return FILTR_ERR_INVALID;
  }
  if (p->affine != 0 && p->affine != 1 && p->affine != FILTR_AFFINE_MID) {
    set_error("affine must be 0, 1 or FILTR_AFFINE_MID");
    return FILTR_ERR_INVALID;
  }
  if (p->gap_extend < 0 || (p->affine && p->gap_open < 0) || p->gap_extend > (1 << 20) ||
      (p->affine && p->gap_open > (1 << 20))) {
    set_error("gap penalties must lie in [0, 2^20]");
    return FILTR_ERR_INVALID;
  }
  if (!p->subst) {
    set_error("subst is NULL");
    return FILTR_ERR_INVALID;
  }
  if (p->prune & ~(uint32_t)(FILTR_PRUNE_BAND | FILTR_PRUNE_XDROP | FILTR_PRUNE_BAND_LITERAL |
                             FILTR_PRUNE_ZDROP | FILTR_PRUNE_XDROP_RUNNING)) {
    set_error("unknown prune bits 0x%x", p->prune);
    return FILTR_ERR_INVALID;
  }
  const bool band = (p->prune & (FILTR_PRUNE_BAND | FILTR_PRUNE_BAND_LITERAL)) != 0;
  const bool zd = (p->prune & FILTR_PRUNE_ZDROP) != 0;
  const bool xd = (p->prune & FILTR_PRUNE_XDROP) != 0 || zd;
  if (zd && (p->prune & FILTR_PRUNE_XDROP)) {
    set_error("FILTR_PRUNE_XDROP and FILTR_PRUNE_ZDROP exclude each other");
    return FILTR_ERR_INVALID;
  }
  const bool mid = p->affine == FILTR_AFFINE_MID;
  if (mid && (zd || (p->prune & FILTR_PRUNE_BAND_LITERAL))) {
    set_error("the M/I/D form runs with X-drop or the widened band, not Z-drop or the literal band");
    return FILTR_ERR_UNSUPPORTED;
  }
  if ((p->prune & FILTR_PRUNE_XDROP_RUNNING) && !xd) {
    set_error("FILTR_PRUNE_XDROP_RUNNING needs FILTR_PRUNE_XDROP or FILTR_PRUNE_ZDROP");
    return FILTR_ERR_INVALID;
  }
  if (band && p->band < 0) {
    set_error("band must be >= 0");
    return FILTR_ERR_INVALID;
  }
  if (xd && p->xdrop < 0) {
    set_error("xdrop must be >= 0");
    return FILTR_ERR_INVALID;
  }
  if (p->traceback != 0 && p->traceback != 1) {
    set_error("traceback must be 0 or 1");
    return FILTR_ERR_INVALID;
  }
  if (p->precision < FILTR_PREC_AUTO || p->precision > FILTR_PREC_I16X2) {
    set_error("unknown precision");
    return FILTR_ERR_INVALID;
  }
  memset(sp, 0, sizeof *sp);
  sp->mode = p->mode;
  sp->affine = p->affine ? 1 : 0;
  sp->o = p->affine ? p->gap_open : 0;
  sp->e = p->gap_extend;
  sp->alphabet = p->alphabet;
  sp->use_band = band ? 1 : 0;
  sp->band_literal = (p->prune & FILTR_PRUNE_BAND_LITERAL) ? 1 : 0;
  sp->band = band ? p->band : 0;
  // the M/I/D form runs on the antidiagonal sweep, without a threshold unless
  // X-drop is asked for
  sp->use_xdrop = (xd || mid) ? 1 : 0;
  sp->zdrop = zd ? 1 : 0;
  sp->xrun = (p->prune & FILTR_PRUNE_XDROP_RUNNING) ? 1 : 0;
  sp->xdrop = xd ? p->xdrop : (mid ? FILTR_XDROP_INF : 0);
  sp->mid = mid ? 1 : 0;
  sp->traceback = p->traceback;
  sp->precision = p->precision;
  sp->smin = 127;
  sp->smax = -128;
  for (int t = 0; t < p->alphabet * p->alphabet; ++t) {
    sp->subst[t] = p->subst[t];
    sp->smin = std::min(sp->smin, (int32_t)p->subst[t]);
    sp->smax = std::max(sp->smax, (int32_t)p->subst[t]);
  }
  // one match score and one mismatch score (DNA +2 / -4): the packed sweep
  // then scores two cells by comparing codes instead of looking them up
  sp->uni = 1;
  sp->uni_match = p->subst[0];
  sp->uni_mismatch = p->alphabet > 1 ? p->subst[1] : 0;
  for (int a = 0; a < p->alphabet; ++a)
    for (int b = 0; b < p->alphabet; ++b)
      if (p->subst[a * p->alphabet + b] != (a == b ? sp->uni_match : sp->uni_mismatch)) sp->uni = 0;
  return FILTR_OK;
}


// ---- workspace carving ------------------------------------------------------
struct Carver {
  char *base;
  size_t cap, used = 0;
  template <class T>
  T *take(size_t count, size_t align = 256) {
    used = (used + align - 1) / align * align;
    T *p = reinterpret_cast<T *>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

int Ctx::full_blocks_per_sm(int R, const ScoreParams &sp) {
  const auto key = std::make_tuple(R, sp.mode, sp.affine, sp.traceback, sp.use_band, sp.alphabet);
  auto it = occ_cache.find(key);
  if (it != occ_cache.end()) return it->second;
  int nb = full_max_blocks_per_sm(R, sp, sp.alphabet);
  if (nb < 1) nb = 1;
  occ_cache[key] = nb;
  return nb;
}

int Ctx::pack_blocks_per_sm(int R, const ScoreParams &sp) {
  const auto key = std::make_tuple(R | 0x100, sp.mode, sp.affine, sp.traceback, 0, sp.alphabet);
  auto it = occ_cache.find(key);
  if (it != occ_cache.end()) return it->second;
  int nb = pack_max_blocks_per_sm(R, sp);
  if (nb < 1) nb = 1;
  occ_cache[key] = nb;
  return nb;
}

int Ctx::graph_blocks_per_sm(int R, bool packed, const ScoreParams &sp) {
  const auto key = std::make_tuple(R | (packed ? 0x300 : 0x200), sp.mode, sp.affine, sp.traceback,
                                   sp.use_band, sp.alphabet);
  auto it = occ_cache.find(key);
  if (it != occ_cache.end()) return it->second;
  int nb = packed ? pack_graph_blocks_per_sm(R, sp) : full_graph_blocks_per_sm(R, sp);
  if (nb < 1) nb = 1;
  occ_cache[key] = nb;
  return nb;
}

cudaEvent_t Ctx::next_event() {
  if (ev_used == ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ev_pool.push_back(e);
  }
  return ev_pool[ev_used++];
}

void Ctx::span_begin(int phase, cudaStream_t st) {
  if (!timing) return;
  Span sp{phase, next_event(), nullptr};
  if (sp.a) cudaEventRecord(sp.a, st);
  spans.push_back(sp);
}

void Ctx::span_end(cudaStream_t st) {
  if (!timing || spans.empty()) return;
  spans.back().b = next_event();
  if (spans.back().b) cudaEventRecord(spans.back().b, st);
}

bool Ctx::ensure_side(int n) {
  if (!fork_ev && cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming) != cudaSuccess) {
    fork_ev = nullptr;
    cudaGetLastError();
    return false;
  }
  while ((int)side.size() < n) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(s);
      cudaGetLastError();
      return false;
    }
    side.push_back(s);
    join_ev.push_back(e);
  }
  return true;
}

bool Ctx::ensure_host(size_t bytes) {
  if (h_stage_bytes >= bytes) return true;
  if (h_stage) cudaFreeHost(h_stage);
  h_stage = nullptr;
  h_stage_bytes = 0;
  size_t want = std::max(bytes, (size_t)1 << 20);
  if (cudaHostAlloc(&h_stage, want, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h_stage_bytes = want;
  return true;
}

// The batched call.  host_* may carry host copies of lengths and offsets
// (the host-buffer entry point has them); otherwise they are read back.
filtr_status align_batch_impl(Ctx *ctx, const filtr_params *params, uint32_t n,
                              const BatchDev &b, filtr_result *out, uint32_t *cigar,
                              uint64_t cap, cudaStream_t st, bool plain,
                              const uint32_t *host_ql, const uint32_t *host_rl,
                              bool prevalidated) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (n == 0) return FILTR_OK;
  if (!b.q_seq || !b.r_seq || !b.q_off || !b.r_off || !b.q_len || !b.r_len || !out) {
    set_error("a batch pointer is NULL");
    return FILTR_ERR_INVALID;
  }
  if (sp.traceback && !cigar && cap > 0) {
    set_error("cigar is NULL but cigar_cap > 0");
    return FILTR_ERR_INVALID;
  }
  // X-drop / Z-drop pairs take the packed sweep when their threshold leaves
  // room in 15 bits (those that leave the range anyway are rerun in int32)
  const Ctx::SweepChoice *swc = sp.use_xdrop ? ctx->sweep_choice(sp) : nullptr;
  sp.xd16 = (ctx->xd16_mode != 1 && xd16_eligible(sp) && (!swc || swc->packed || ctx->xd16_mode == 2))
                ? 1
                : 0;
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
  if (ctx->done_ev) {
    ce = cudaEventSynchronize(ctx->done_ev);  // the previous call is finished with the workspace
    if (ce != cudaSuccess) return cuda_fail(ce, "waiting for the previous call");
  }
  ctx->ev_used = 0;
  ctx->spans.clear();
  uint32_t launches = 0;

  // 1. workspace parts whose size depends on n only
  Carver c{ctx->ws, ctx->ws_bytes};
  DevPlanState *d_ps = c.take<DevPlanState>(1);
  uint32_t *d_bad = reinterpret_cast<uint32_t *>(  // residue validation count (bad[0])
      reinterpret_cast<char *>(d_ps) + offsetof(DevPlanState, bad));
  uint32_t *d_order = c.take<uint32_t>(n);
  TbLayout *d_tbl = c.take<TbLayout>(n);
  uint64_t *d_stage_off = c.take<uint64_t>(n);
  FwdOut *d_fwd = c.take<FwdOut>(n);
  uint64_t *d_offs = c.take<uint64_t>(n);
  const size_t n_counters = (size_t)n + 4096;
  uint32_t *d_counters = c.take<uint32_t>(n_counters);
  uint64_t *d_total = c.take<uint64_t>(4);
  uint32_t *d_ovf = c.take<uint32_t>(n);
  uint32_t *d_novf = c.take<uint32_t>(8);  // [0] window overflows, [4] packed-range overflows
  uint32_t *d_ovf16 = sp.xd16 ? c.take<uint32_t>(n) : nullptr;
  uint32_t *d_rerun = c.take<uint32_t>(n);
  // The device planner serves tiled batches (not X-drop, not one launch per
  // pair) once planning on the host would cost more than the read-back: when
  // the lengths must come back anyway, from a few hundred pairs; otherwise
  // (host lengths, already validated) from a few thousand.
  const bool must_sync = !(prevalidated && host_ql);
  bool dev_plan = !plain && !sp.use_xdrop &&
                  (ctx->dev_plan_mode == 2 ||
                   (ctx->dev_plan_mode == 0 && n >= (must_sync ? 256u : 4096u)));
  const uint32_t plan_blocks = (n + DEV_PLAN_BLOCK - 1) / DEV_PLAN_BLOCK;
  uint16_t *d_pkey = dev_plan ? c.take<uint16_t>(n) : nullptr;
  uint64_t *d_pwords = dev_plan ? c.take<uint64_t>(n) : nullptr;
  uint64_t *d_pblk = dev_plan ? c.take<uint64_t>(plan_blocks) : nullptr;
  if (c.used > ctx->ws_bytes) {
    set_error("workspace of %zu bytes is too small for this batch's fixed buffers (%zu bytes)",
              ctx->ws_bytes, c.used);
    return FILTR_ERR_NOMEM;
  }
  const ShapeCost *costs = ctx->tuned_costs(sp);
  if (!costs) costs = kDefaultShapeCost;

  // 2. residue validation, the device plan, and the lengths or the plan's
  // totals back to the host (one synchronisation)
  const size_t head_bytes = offsetof(DevPlanState, hist);
  const size_t lens_bytes = (size_t)n * 4 * 2;
  if (!ctx->ensure_host(head_bytes + lens_bytes + 64)) {
    set_error("pinned host allocation of %zu bytes failed", head_bytes + lens_bytes);
    return FILTR_ERR_NOMEM;
  }
  DevPlanState *h_ps = reinterpret_cast<DevPlanState *>(ctx->h_stage);  // bad[] and sum only
  uint32_t *h_ql = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ctx->h_stage) +
                                                (head_bytes + 255) / 256 * 256);
  uint32_t *h_rl = h_ql + n;
  memset(h_ps, 0, head_bytes);
  using clk = std::chrono::steady_clock;
  const auto ms_since = [](clk::time_point t) {
    return std::chrono::duration<double, std::milli>(clk::now() - t).count();
  };
  ctx->last_host_wait_ms = ctx->last_host_plan_ms = 0;
  ce = cudaMemsetAsync(d_ps, 0, sizeof(DevPlanState), st);
  if (ce != cudaSuccess) return cuda_fail(ce, "clearing the plan state");
  if (!prevalidated) {
    ctx->span_begin(Ctx::PH_VALIDATE, st);
    ce = launch_validate_pairs(b, n, sp.alphabet, d_bad, st);
    ctx->span_end(st);
    ++launches;
  }
  DevPlanArgs pa{};
  if (dev_plan && ce == cudaSuccess) {
    pa.q_len = b.q_len;
    pa.r_len = b.r_len;
    pa.n = n;
    pa.sp = sp;
    pa.tab = make_shape_table(costs, sp);
    pa.state = d_ps;
    pa.key = d_pkey;
    pa.words = d_pwords;
    pa.blk = d_pblk;
    pa.order = d_order;
    pa.tbl = d_tbl;
    pa.stage_off = d_stage_off;
    ce = launch_plan(pa, st);
    launches += 3;
  }
  if (must_sync || dev_plan) {
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_ps, d_ps, head_bytes, cudaMemcpyDeviceToHost, st);
    if (!host_ql && !dev_plan) {
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_ql, b.q_len, n * 4, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_rl, b.r_len, n * 4, cudaMemcpyDeviceToHost, st);
    }
    const auto t_wait = clk::now();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    ctx->last_host_wait_ms = ms_since(t_wait);
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "validation and planning");
  const auto t_plan = clk::now();
  if (h_ps->bad[0]) {
    set_error("%u residue codes are >= the alphabet size %d", h_ps->bad[0], sp.alphabet);
    return FILTR_ERR_INVALID;
  }
  const DevPlanSummary dsum = h_ps->sum;  // the staging area is reused below

  // 3. sizes, then the workspace parts that depend on them
  uint64_t max_m = 0, max_n = 0, stage_words = 0;
  if (dev_plan) {
    max_m = dsum.max_m;
    max_n = dsum.max_n;
    stage_words = dsum.stage_words;
  } else {
    if (host_ql) {
      memcpy(h_ql, host_ql, n * 4);
      memcpy(h_rl, host_rl, n * 4);
    }
    for (uint32_t p = 0; p < n; ++p) {
      max_m = std::max<uint64_t>(max_m, h_ql[p]);
      max_n = std::max<uint64_t>(max_n, h_rl[p]);
      if (sp.traceback) stage_words += (uint64_t)h_ql[p] + h_rl[p] + 1;
    }
  }
  if (max_m >= (1u << 30) || max_n >= (1u << 30)) {
    set_error("sequence longer than 2^30");
    return FILTR_ERR_UNSUPPORTED;
  }
  if (!score_range_ok(sp, max_m, max_n)) {
    set_error("scores could exceed 2^28 (2^26 for local alignments) for these lengths and penalties");
    return FILTR_ERR_UNSUPPORTED;
  }
  int blocks_per_sm = 1;
  for (int R : {8, 16, 24, 32}) blocks_per_sm = std::max(blocks_per_sm, ctx->full_blocks_per_sm(R, sp));
  if (!sp.use_band && !sp.use_xdrop && sp.precision != FILTR_PREC_I32)
    for (int k = 0; k < SHAPE_TILED; ++k)
      if (kDefaultShapeCost[k].packed)
        blocks_per_sm = std::max(blocks_per_sm, ctx->pack_blocks_per_sm(kDefaultShapeCost[k].R, sp));
  const int grid_max = plain ? 1 : (int)std::min<int64_t>((int64_t)ctx->sms * blocks_per_sm,
                                                          ((int64_t)n + FULL_WARPS - 1) / FULL_WARPS);
  const uint32_t strip_stride = (uint32_t)(max_n + 2);
  // Strip buffers: one region for launches in sequence; when the device plan
  // gives pairs to several tiled shapes, their launches run concurrently on
  // side streams (one launch's tail overlaps the others' work), each shape
  // with its own region.
  size_t strip_elems = (size_t)grid_max * FULL_WARPS * strip_stride;
  size_t shape_strip[SHAPE_TILED] = {};
  int shape_grid[SHAPE_TILED] = {};
  int n_conc = 0;
  if (dev_plan) {
    size_t tot = 0;
    for (int k = 0; k < SHAPE_TILED; ++k) {
      if (!dsum.count[k]) continue;
      const int bps = costs[k].packed ? ctx->pack_blocks_per_sm(costs[k].R, sp)
                                      : ctx->full_blocks_per_sm(costs[k].R, sp);
      shape_grid[k] = (int)std::min<int64_t>((int64_t)ctx->sms * bps,
                                             ((int64_t)dsum.count[k] + FULL_WARPS - 1) / FULL_WARPS);
      shape_strip[k] = tot;
      tot += (size_t)shape_grid[k] * FULL_WARPS * strip_stride;
      ++n_conc;
    }
    if (n_conc >= 2 && ctx->ensure_side(n_conc))
      strip_elems = std::max(strip_elems, tot);
    else
      n_conc = 0;
  }
  int2 *d_strip = c.take<int2>(strip_elems);
  uint32_t *d_stage = sp.traceback ? c.take<uint32_t>(stage_words) : nullptr;
  uint32_t *d_tb = c.take<uint32_t>(0);
  if (c.used > ctx->ws_bytes) {
    set_error("workspace of %zu bytes is too small for this batch's fixed buffers (%zu bytes)",
              ctx->ws_bytes, c.used);
    return FILTR_ERR_NOMEM;
  }
  const uint64_t tb_budget = (ctx->ws_bytes - c.used) / 4;

  // 4. the plan: the device's when its traceback fits one wave, else the host's
  Plan &P = ctx->plan;
  uint32_t n_main = 0, n_trivial = 0;
  if (dev_plan && (!sp.traceback || dsum.tb_words <= tb_budget)) {
    P.waves.clear();
    P.trivial.clear();
    Wave w;
    w.tb_words = dsum.tb_words;
    uint32_t at = 0;
    for (int k = 0; k < SHAPE_TILED; ++k) {
      if (!dsum.count[k]) continue;
      Group g;
      g.family = costs[k].packed ? FAM_PACK : FAM_FULL;
      g.R = (uint8_t)costs[k].R;
      g.warps = 1;
      g.shape = (int8_t)k;
      g.begin = at;
      g.end = at + dsum.count[k];
      at = g.end;
      w.groups.push_back(g);
    }
    n_main = at;
    n_trivial = dsum.count[KEY_TRIVIAL];
    w.walk_begin = 0;
    w.walk_end = n_main;
    if (n_main) P.waves.push_back(w);
    P.cigar_upper = dsum.cigar_upper;
    P.cells_estimate = dsum.cells;
    P.cells_packed = dsum.cells_packed;
    P.xdrop_w0 = 1;
    ce = cudaMemsetAsync(d_counters, 0, n_counters * 4, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "clearing the work queues");
  } else {
    if (dev_plan && !host_ql) {  // the host plan needs the lengths after all
      ce = cudaMemcpyAsync(h_ql, b.q_len, n * 4, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_rl, b.r_len, n * 4, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) return cuda_fail(ce, "reading lengths");
    } else if (dev_plan) {
      memcpy(h_ql, host_ql, n * 4);
      memcpy(h_rl, host_rl, n * 4);
    }
    dev_plan = false;
    n_conc = 0;
    ctx->h_ql.assign(h_ql, h_ql + n);  // the staging area is reused for the plan upload
    ctx->h_rl.assign(h_rl, h_rl + n);
    // first group width of X-drop pairs: the test hook's, the tuned one, or the
    // planner's estimate from the expected live width
    const int w0 = ctx->xdrop_warps0 > 0 ? ctx->xdrop_warps0 : (swc ? swc->warps : 0);
    PlanInput in{&sp, n, ctx->h_ql.data(), ctx->h_rl.data(), tb_budget, 8, w0};
    in.shape_cost = costs;
    if (!make_plan(in, &P)) return FILTR_ERR_NOMEM;
    n_main = (uint32_t)P.order.size();
    n_trivial = (uint32_t)P.trivial.size();
    const size_t up_bytes = n * (4 + sizeof(TbLayout) + 8) + 64;
    if (!ctx->ensure_host(up_bytes + 64)) {
      set_error("pinned host allocation failed");
      return FILTR_ERR_NOMEM;
    }
    char *hs = reinterpret_cast<char *>(ctx->h_stage);
    memcpy(hs, P.order.data(), (size_t)n_main * 4);  // then the trivial pairs
    if (n_trivial) memcpy(hs + (size_t)n_main * 4, P.trivial.data(), (size_t)n_trivial * 4);
    memcpy(hs + n * 4, P.tbl.data(), n * sizeof(TbLayout));
    memcpy(hs + n * (4 + sizeof(TbLayout)), P.stage_off.data(), n * 8);
    ce = cudaMemcpyAsync(d_order, hs, n * 4, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_tbl, hs + n * 4, n * sizeof(TbLayout), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_stage_off, hs + n * (4 + sizeof(TbLayout)), n * 8, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d_counters, 0, n_counters * 4, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "uploading the plan");
  }
  ctx->last_dev_plan = dev_plan;
  const std::vector<uint32_t> &ql = ctx->h_ql, &rl = ctx->h_rl;
  ctx->last_host_plan_ms = ms_since(t_plan);

  FullArgs fa;
  fa.b = b;
  fa.sp = sp;
  fa.out = out;
  fa.fwd = d_fwd;
  fa.tb = d_tb;
  fa.tbl = d_tbl;
  fa.strip_buf = d_strip;
  fa.strip_stride = strip_stride;
  fa.max_n = 0;
  fa.max_m = 0;
  fa.ck = nullptr;
  fa.ovf16 = d_ovf16;
  fa.n_ovf16 = d_novf + 4;
  fa.x16_rebase = ctx->xd16_mode == 2 ? 0 : X16_REBASE;
  WalkArgs wa;
  wa.b = b;
  wa.sp = sp;
  wa.out = out;
  wa.fwd = d_fwd;
  wa.tb = d_tb;
  wa.tbl = d_tbl;
  wa.stage = d_stage;
  wa.stage_off = d_stage_off;

  // 4. waves.  X-drop pairs whose live region outgrows their window come back
  // through the overflow list and are rerun with a wider group (1 -> 4 -> 16
  // warps) once the wave's walk is done with the traceback area.
  size_t counter_i = 0;
  auto run_group = [&](const uint32_t *d_ord, uint32_t cnt, uint8_t family, int R, int W,
                       cudaStream_t gs, int grid_cap) -> bool {
    if (cnt == 0) return true;
    if (family == FAM_FULL || family == FAM_PACK) {
      const bool pk = family == FAM_PACK;
      if (plain) {
        for (uint32_t t = 0; t < cnt; ++t) {
          fa.order = d_ord + t;
          fa.n_order = 1;
          fa.counter = d_counters + (counter_i++ % n_counters);
          ce = pk ? launch_pack(fa, R, 1, st) : launch_full(fa, R, 1, st);
          ++launches;
          if (ce != cudaSuccess) return false;
          if (sp.traceback) {
            wa.order = fa.order;
            wa.n_order = 1;
            ce = launch_walk(wa, st);
            ++launches;
            if (ce != cudaSuccess) return false;
          }
        }
        return true;
      }
      fa.order = d_ord;
      fa.n_order = cnt;
      fa.counter = d_counters + (counter_i++ % n_counters);
      const int bps = pk ? ctx->pack_blocks_per_sm(R, sp) : ctx->full_blocks_per_sm(R, sp);
      // the strip buffer region holds grid_cap blocks' warps
      int grid = (int)std::min<int64_t>((int64_t)ctx->sms * bps, (cnt + FULL_WARPS - 1) / FULL_WARPS);
      grid = std::min(grid, grid_cap);
      ce = pk ? launch_pack(fa, R, std::max(grid, 1), gs) : launch_full(fa, R, std::max(grid, 1), gs);
      ++launches;
      return ce == cudaSuccess;
    }
    if (plain) {
      for (uint32_t t = 0; t < cnt; ++t) {
        fa.order = d_ord + t;
        fa.n_order = 1;
        fa.counter = d_counters + (counter_i++ % n_counters);
        ce = launch_xdrop(fa, W, 1, d_ovf, d_novf, st);
        ++launches;
        if (ce != cudaSuccess) return false;
        if (sp.traceback) {  // a pair that outgrew its window is skipped by the walk
          wa.order = fa.order;
          wa.n_order = 1;
          ce = launch_walk_xd(wa, st);
          ++launches;
          if (ce != cudaSuccess) return false;
        }
      }
      return true;
    }
    fa.order = d_ord;
    fa.n_order = cnt;
    fa.counter = d_counters + (counter_i++ % n_counters);
    const int ppc = xd_pairs_per_cta(W, fa.sp);
    const int bps = std::max(1, xd_max_blocks_per_sm(W, fa.sp));
    int grid = (int)std::min<int64_t>((int64_t)ctx->sms * bps, (cnt + ppc - 1) / ppc);
    ce = launch_xdrop(fa, W, std::max(grid, 1), d_ovf, d_novf, st);
    ++launches;
    return ce == cudaSuccess;
  };
  // pairs that outgrew their window (list) and, from the packed sweep, pairs
  // that left its 16-bit range (list16); both counters come back in one copy
  auto read_overflow = [&](std::vector<uint32_t> *list, std::vector<uint32_t> *list16) -> bool {
    uint32_t *h = reinterpret_cast<uint32_t *>(ctx->h_stage);
    ce = cudaMemcpyAsync(h, d_novf, 32, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return false;
    const uint32_t k = h[0], k16 = fa.sp.xd16 ? h[4] : 0;
    list->clear();
    if (k) {
      ce = cudaMemcpyAsync(h, d_ovf, k * 4ull, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) return false;
      list->assign(h, h + k);
    }
    if (k16) {
      ce = cudaMemcpyAsync(h, d_ovf16, k16 * 4ull, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) return false;
      list16->insert(list16->end(), h, h + k16);
    }
    return true;
  };
  auto walk = [&](const uint32_t *d_ord, uint32_t cnt) -> bool {
    if (!sp.traceback || plain || cnt == 0) return true;
    wa.order = d_ord;
    wa.n_order = cnt;
    ctx->span_begin(Ctx::PH_WALK, st);
    ce = sp.use_xdrop ? launch_walk_xd(wa, st) : launch_walk(wa, st);
    ctx->span_end(st);
    ++launches;
    return ce == cudaSuccess;
  };
  std::vector<uint32_t> pending, pending16;
  for (const Wave &w : P.waves) {
    bool has_xd = false;
    ctx->span_begin(Ctx::PH_FORWARD, st);
    for (const Group &g : w.groups) has_xd |= g.family == FAM_XDROP;
    if (has_xd) {
      ce = cudaMemsetAsync(d_novf, 0, 32, st);
      if (ce != cudaSuccess) return cuda_fail(ce, "overflow reset");
    }
    if (n_conc) {  // fork: each shape on its own side stream and strip region; join on st
      ce = cudaEventRecord(ctx->fork_ev, st);
      int si = 0;
      for (const Group &g : w.groups) {
        if (ce != cudaSuccess) break;
        cudaStream_t s2 = ctx->side[si];
        ce = cudaStreamWaitEvent(s2, ctx->fork_ev, 0);
        fa.strip_buf = d_strip + shape_strip[g.shape];
        if (ce == cudaSuccess &&
            !run_group(d_order + g.begin, g.end - g.begin, g.family, g.R, g.warps, s2,
                       shape_grid[g.shape]))
          return cuda_fail(ce, "forward kernel launch");
        if (ce == cudaSuccess) ce = cudaEventRecord(ctx->join_ev[si], s2);
        ++si;
      }
      for (int i = 0; i < si && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(st, ctx->join_ev[i], 0);
      fa.strip_buf = d_strip;
      if (ce != cudaSuccess) return cuda_fail(ce, "forking the forward launches");
    } else {
      for (const Group &g : w.groups)
        if (!run_group(d_order + g.begin, g.end - g.begin, g.family, g.R, g.warps, st, grid_max))
          return cuda_fail(ce, "forward kernel launch");
    }
    ctx->span_end(st);
    std::vector<uint32_t> ovf;
    if (has_xd && !read_overflow(&ovf, &pending16)) return cuda_fail(ce, "reading the overflow list");
    if (!walk(d_order + w.walk_begin, w.walk_end - w.walk_begin)) return cuda_fail(ce, "walk launch");
    pending.insert(pending.end(), ovf.begin(), ovf.end());
  }
  const uint32_t n_xd16 = fa.sp.xd16 ? n_main : 0;
  uint32_t n_xd16_rerun = 0;
  // rerun `todo` at group width W, in sub-waves that fit the traceback budget;
  // pairs that outgrow the window again join `pending`, pairs that leave the
  // packed range join `pending16`
  auto rerun = [&](std::vector<uint32_t> &todo, int W) -> bool {
    size_t i0 = 0;
    while (i0 < todo.size()) {
      size_t i1 = i0;
      uint64_t used = 0;
      while (i1 < todo.size()) {
        const uint32_t p = todo[i1];
        const uint64_t words = sp.traceback ? xd_tb_words(ql[p], rl[p], W, 8) : 0;
        if (used + words > tb_budget) break;
        TbLayout &L = P.tbl[p];
        L.off = used;
        L.warps = (uint8_t)W;
        used += words;
        ++i1;
      }
      if (i1 == i0) {  // a single pair does not fit: it keeps status TOO_WIDE
        ++i0;
        continue;
      }
      const uint32_t cnt = (uint32_t)(i1 - i0);
      char *h = reinterpret_cast<char *>(ctx->h_stage);
      memcpy(h, todo.data() + i0, cnt * 4);
      memcpy(h + n * 4ull, P.tbl.data(), n * sizeof(TbLayout));
      ce = cudaMemcpyAsync(d_rerun, h, cnt * 4ull, cudaMemcpyHostToDevice, st);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_tbl, h + n * 4ull, n * sizeof(TbLayout), cudaMemcpyHostToDevice, st);
      if (ce == cudaSuccess) ce = cudaMemsetAsync(d_novf, 0, 32, st);
      if (ce != cudaSuccess) return false;
      ctx->span_begin(Ctx::PH_FORWARD, st);
      if (!run_group(d_rerun, cnt, FAM_XDROP, 8, W, st, grid_max)) return false;
      ctx->span_end(st);
      std::vector<uint32_t> ovf;
      if (!read_overflow(&ovf, &pending16)) return false;
      if (!walk(d_rerun, cnt)) return false;
      pending.insert(pending.end(), ovf.begin(), ovf.end());
      i0 = i1;
    }
    return true;
  };
  static const int kWider[] = {2, 4, 8, 16, 32};
  auto ladder = [&](int w_done) -> bool {  // rerun `pending` ever wider, above w_done warps
    for (int wi = 0; wi < 5 && !pending.empty(); ++wi) {
      const int W = kWider[wi];
      if (W <= w_done) continue;
      std::vector<uint32_t> todo;
      todo.swap(pending);
      if (!rerun(todo, W)) return false;
    }
    return true;
  };
  if (!ladder(P.xdrop_w0)) return cuda_fail(ce, "rerun");
  if (!pending16.empty()) {  // pairs that left the packed range: the int32 sweep
    std::vector<uint32_t> todo;
    todo.swap(pending16);
    n_xd16_rerun = (uint32_t)todo.size();
    fa.sp.xd16 = 0;
    const int w0 = std::max(1, (int)P.xdrop_w0);
    if (!rerun(todo, w0) || !ladder(w0)) return cuda_fail(ce, "int32 rerun");
  }
  if (n_trivial) {
    ce = launch_trivial(b, sp, d_order + n_main, n_trivial, out, d_fwd, st);
    ++launches;
    if (ce == cudaSuccess && sp.traceback) {
      wa.order = d_order + n_main;
      wa.n_order = n_trivial;
      ce = launch_walk(wa, st);
      ++launches;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "empty-pair launch");
  }

  // 5. CIGAR placement
  if (sp.traceback) {
    ctx->span_begin(Ctx::PH_PLACE, st);
    ce = launch_scan_offsets(out, n, d_offs, d_total, st);
    if (ce == cudaSuccess) ce = launch_compact(wa, n, d_offs, cigar, cap, out, st);
    ctx->span_end(st);
    launches += 2;
    if (ce != cudaSuccess) return cuda_fail(ce, "CIGAR placement");
    if (cap < P.cigar_upper) {
      uint64_t *h_total = reinterpret_cast<uint64_t *>(ctx->h_stage);
      ce = cudaMemcpyAsync(h_total, d_total, 8, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) return cuda_fail(ce, "reading the CIGAR total");
      if (*h_total > cap) {
        set_error("CIGARs need %llu ops, cigar_cap is %llu", (unsigned long long)*h_total,
                  (unsigned long long)cap);
        ctx->last_launches = launches;
        return FILTR_ERR_CIGAR_CAP;
      }
    }
  }
  ctx->last_cells_estimate = P.cells_estimate;
  ctx->last_cells_packed = P.cells_packed;
  ctx->last_xd16 = n_xd16;
  ctx->last_xd16_rerun = n_xd16_rerun;
  ctx->last_pairs_packed = 0;
  for (const Wave &w : P.waves)
    for (const Group &g : w.groups)
      if (g.family == FAM_PACK) ctx->last_pairs_packed += g.end - g.begin;
  ctx->last_waves = (int)P.waves.size();
  ctx->last_launches = launches;
  if (!ctx->done_ev) cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
  if (ctx->done_ev) cudaEventRecord(ctx->done_ev, st);
  return FILTR_OK;
}

}  // namespace filtr

using namespace filtr;

extern "C" {

const char *filtr_last_error(void) { return g_err.c_str(); }

const char *filtr_version(void) { return "filtr-gb300 0.1 (sm_103a)"; }

filtr_status filtr_params_check(const filtr_params *params) {
  ScoreParams sp;
  return to_score_params(params, &sp);
}

filtr_status filtr_test_plan_host(const filtr_params *params, uint32_t n, const uint32_t *q_len,
                                  const uint32_t *r_len, uint64_t tb_budget_words, uint32_t *order,
                                  uint32_t *wave, uint64_t *tb_off, uint64_t *tb_words,
                                  uint32_t *kernel, uint64_t *wave_info, uint32_t *counts) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (!counts || (n && (!q_len || !r_len || !order || !wave || !tb_off || !tb_words || !kernel ||
                        !wave_info))) {
    set_error("filtr_test_plan_host: NULL argument");
    return FILTR_ERR_INVALID;
  }
  PlanInput in{&sp, n, q_len, r_len, tb_budget_words, 8, 0};
  Plan P;
  if (!make_plan(in, &P)) return FILTR_ERR_NOMEM;
  const uint32_t nm = (uint32_t)P.order.size(), nt = (uint32_t)P.trivial.size();
  for (uint32_t t = 0; t < nm; ++t) order[t] = P.order[t];
  for (uint32_t t = 0; t < nt; ++t) order[nm + t] = P.trivial[t];
  for (uint32_t p = 0; p < n; ++p) {
    wave[p] = UINT32_MAX;
    tb_off[p] = tb_words[p] = 0;
    kernel[p] = 0;
  }
  for (size_t w = 0; w < P.waves.size(); ++w) {
    const Wave &W = P.waves[w];
    wave_info[3 * w] = W.tb_words;
    wave_info[3 * w + 1] = W.walk_begin;
    wave_info[3 * w + 2] = W.walk_end;
    for (const Group &g : W.groups)
      for (uint32_t t = g.begin; t < g.end; ++t) {
        const uint32_t p = P.order[t];
        wave[p] = (uint32_t)w;
        kernel[p] = (uint32_t)g.family << 16 | (uint32_t)g.R << 8 | g.warps;
        tb_off[p] = P.tbl[p].off;
        tb_words[p] = sp.traceback ? P.s_words[p] : 0;
      }
  }
  counts[0] = nm;
  counts[1] = (uint32_t)P.waves.size();
  counts[2] = nt;
  return FILTR_OK;
}

filtr_status filtr_ctx_create(int device, size_t workspace_bytes, filtr_ctx **out) {
  if (!out) {
    set_error("out is NULL");
    return FILTR_ERR_INVALID;
  }
  *out = nullptr;
  Ctx *c = nullptr;
  filtr_status rc = filtr::ctx_new(device, workspace_bytes, &c);
  if (rc == FILTR_OK) *out = reinterpret_cast<filtr_ctx *>(c);
  return rc;
}

filtr_status filtr_ctx_destroy(filtr_ctx *ctx) {
  filtr::ctx_delete(reinterpret_cast<Ctx *>(ctx));
  return FILTR_OK;
}

}  // extern "C"

namespace filtr {

filtr_status ctx_new(int device, size_t workspace_bytes, Ctx **out) {
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) {
    set_error("device %d out of range (%d devices)", device, ndev);
    return FILTR_ERR_INVALID;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  Ctx *c = new (std::nothrow) Ctx();
  if (!c) {
    set_error("host allocation failed");
    return FILTR_ERR_NOMEM;
  }
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  size_t ws = workspace_bytes ? workspace_bytes : ((size_t)8 << 30);
  if (!workspace_bytes && ws > fr / 2) ws = fr / 2;
  e = cudaMalloc(&c->ws, ws);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_error("cudaMalloc of a %zu-byte workspace failed", ws);
    return FILTR_ERR_NOMEM;
  }
  c->ws_bytes = ws;
  e = cudaMalloc(&c->d_small, 4096);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->ws);
    delete c;
    set_error("cudaMalloc of 4 KiB failed");
    return FILTR_ERR_NOMEM;
  }
  e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return cuda_fail(e, "cudaStreamCreate");
  }
  *out = c;
  return FILTR_OK;
}

void ctx_delete(Ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->own_stream);
  if (c->done_ev) {
    cudaEventSynchronize(c->done_ev);
    cudaEventDestroy(c->done_ev);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaStream_t s : c->side) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : c->join_ev) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->ws) cudaFree(c->ws);
  if (c->d_small) cudaFree(c->d_small);
  if (c->d_io) cudaFree(c->d_io);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  cudaStreamDestroy(c->own_stream);
  delete c;
}

}  // namespace filtr

extern "C" {

filtr_status filtr_pack(const uint8_t *codes, uint64_t n, int32_t alphabet, uint32_t *packed,
                        uint32_t *bad_out, void *stream) {
  if (alphabet != FILTR_ALPHA_DNA && alphabet != FILTR_ALPHA_PROTEIN) {
    set_error("alphabet must be 4 or 20");
    return FILTR_ERR_INVALID;
  }
  if (n && (!codes || !packed || !bad_out)) {
    set_error("NULL pointer");
    return FILTR_ERR_INVALID;
  }
  if (reinterpret_cast<uintptr_t>(codes) & 15u) {
    set_error("filtr_pack: codes must start on a 16-byte boundary (they are read 16 at a time)");
    return FILTR_ERR_INVALID;
  }
  if (reinterpret_cast<uintptr_t>(packed) & 3u) {
    set_error("filtr_pack: packed must start on a 4-byte boundary");
    return FILTR_ERR_INVALID;
  }
  cudaError_t e = launch_pack(codes, n, alphabet, packed, bad_out, (cudaStream_t)stream);
  return e == cudaSuccess ? FILTR_OK : cuda_fail(e, "pack launch");
}

filtr_status filtr_align_batch(filtr_ctx *ctx, const filtr_params *params, uint32_t n_pairs,
                               const uint8_t *q_seq, const uint64_t *q_off, const uint32_t *q_len,
                               const uint8_t *r_seq, const uint64_t *r_off, const uint32_t *r_len,
                               filtr_result *out, uint32_t *cigar, uint64_t cigar_cap,
                               void *stream) {
  if (!ctx) {
    set_error("ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  BatchDev b{q_seq, r_seq, q_off, r_off, q_len, r_len};
  return align_batch_impl(reinterpret_cast<Ctx *>(ctx), params, n_pairs, b, out, cigar, cigar_cap,
                          (cudaStream_t)stream, false, nullptr, nullptr, false);
}

filtr_status filtr_align_batch_plain(filtr_ctx *ctx, const filtr_params *params,
                                     uint32_t n_pairs, const uint8_t *q_seq,
                                     const uint64_t *q_off, const uint32_t *q_len,
                                     const uint8_t *r_seq, const uint64_t *r_off,
                                     const uint32_t *r_len, filtr_result *out, uint32_t *cigar,
                                     uint64_t cigar_cap, void *stream) {
  if (!ctx) {
    set_error("ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  BatchDev b{q_seq, r_seq, q_off, r_off, q_len, r_len};
  return align_batch_impl(reinterpret_cast<Ctx *>(ctx), params, n_pairs, b, out, cigar, cigar_cap,
                          (cudaStream_t)stream, true, nullptr, nullptr, false);
}

filtr_status filtr_align_batch_host(filtr_ctx *ctx, const filtr_params *params, uint32_t n,
                                    const uint8_t *q_seq, const uint64_t *q_off,
                                    const uint32_t *q_len, const uint8_t *r_seq,
                                    const uint64_t *r_off, const uint32_t *r_len,
                                    filtr_result *out, uint32_t *cigar, uint64_t cigar_cap) {
  if (!ctx) {
    set_error("ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  if (n == 0) return FILTR_OK;
  if (!q_seq || !q_off || !q_len || !r_seq || !r_off || !r_len || !out) {
    set_error("a host pointer is NULL");
    return FILTR_ERR_INVALID;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaSetDevice(c->device);
  uint64_t qbytes = 0, rbytes = 0;
  for (uint32_t p = 0; p < n; ++p) {
    qbytes = std::max<uint64_t>(qbytes, q_off[p] + q_len[p]);
    rbytes = std::max<uint64_t>(rbytes, r_off[p] + r_len[p]);
  }
  const bool tb = params && params->traceback;
  const uint64_t ccap = tb ? cigar_cap : 0;
  auto al = [](uint64_t x) { return (x + 255) / 256 * 256; };
  const uint64_t need = al(qbytes) + al(rbytes) + 2 * al(n * 8ull) + 2 * al(n * 4ull) +
                        al(n * sizeof(filtr_result)) + al(ccap * 4);
  if (c->d_io_bytes < need) {
    if (c->d_io) cudaFree(c->d_io);
    c->d_io = nullptr;
    c->d_io_bytes = 0;
    if (cudaMalloc(&c->d_io, need) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %llu bytes for host-buffer staging failed",
                (unsigned long long)need);
      return FILTR_ERR_NOMEM;
    }
    c->d_io_bytes = need;
  }
  char *d = reinterpret_cast<char *>(c->d_io);
  uint8_t *dq = reinterpret_cast<uint8_t *>(d);
  d += al(qbytes);
  uint8_t *dr = reinterpret_cast<uint8_t *>(d);
  d += al(rbytes);
  uint64_t *dqo = reinterpret_cast<uint64_t *>(d);
  d += al(n * 8ull);
  uint64_t *dro = reinterpret_cast<uint64_t *>(d);
  d += al(n * 8ull);
  uint32_t *dql = reinterpret_cast<uint32_t *>(d);
  d += al(n * 4ull);
  uint32_t *drl = reinterpret_cast<uint32_t *>(d);
  d += al(n * 4ull);
  filtr_result *dout = reinterpret_cast<filtr_result *>(d);
  d += al(n * sizeof(filtr_result));
  uint32_t *dcig = ccap ? reinterpret_cast<uint32_t *>(d) : nullptr;
  cudaStream_t st = c->own_stream;
  cudaError_t e = cudaMemcpyAsync(dq, q_seq, qbytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, r_seq, rbytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dqo, q_off, n * 8ull, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dro, r_off, n * 8ull, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dql, q_len, n * 4ull, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(drl, r_len, n * 4ull, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copies");
  BatchDev b{dq, dr, dqo, dro, dql, drl};
  filtr_status rc = align_batch_impl(c, params, n, b, dout, dcig, ccap, st, false, q_len, r_len, false);
  if (rc != FILTR_OK && rc != FILTR_ERR_CIGAR_CAP) return rc;
  e = cudaMemcpyAsync(out, dout, n * sizeof(filtr_result), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy of results");
  if (rc == FILTR_OK && tb && cigar) {
    uint64_t total = 0;
    for (uint32_t p = 0; p < n; ++p) total = std::max<uint64_t>(total, out[p].cigar_off + out[p].cigar_len);
    if (total) {
      e = cudaMemcpyAsync(cigar, dcig, total * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy of CIGARs");
    }
  }
  return rc;
}

filtr_status filtr_ctx_set_timing(filtr_ctx *ctx, int enable) {
  if (!ctx) {
    set_error("ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->timing = enable != 0;
  return FILTR_OK;
}

filtr_status filtr_ctx_last_stats(filtr_ctx *ctx, filtr_stats *out) {
  if (!ctx || !out) {
    set_error("NULL argument");
    return FILTR_ERR_INVALID;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  memset(out, 0, sizeof *out);
  out->launches = c->last_launches;
  out->waves = (uint32_t)c->last_waves;
  out->cells_planned = c->last_cells_estimate;
  out->pairs_i16x2 = c->last_pairs_packed;
  out->cells_i16x2 = c->last_cells_packed;
  out->pairs_xd16 = c->last_xd16;
  out->pairs_xd16_rerun = c->last_xd16_rerun;
  out->device_plan = c->last_dev_plan ? 1u : 0u;
  out->ms_host_wait = c->last_host_wait_ms;
  out->ms_host_plan = c->last_host_plan_ms;
  cudaSetDevice(c->device);
  double *acc[4] = {&out->ms_validate, &out->ms_forward, &out->ms_walk, &out->ms_place};
  cudaEvent_t first = nullptr, last = nullptr;
  for (const auto &sp : c->spans) {
    if (!sp.a || !sp.b) continue;
    cudaError_t e = cudaEventSynchronize(sp.b);
    if (e != cudaSuccess) return cuda_fail(e, "timing event");
    float ms = 0;
    cudaEventElapsedTime(&ms, sp.a, sp.b);
    *acc[sp.phase] += ms;
    if (!first) first = sp.a;
    last = sp.b;
  }
  if (first && last) {
    float ms = 0;
    cudaEventElapsedTime(&ms, first, last);
    out->ms_total = ms;
  }
  return FILTR_OK;
}

filtr_status filtr_probe_int_peak(filtr_ctx *ctx, double out[5]) {
  if (!ctx || !out) {
    set_error("NULL argument");
    return FILTR_ERR_INVALID;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaSetDevice(c->device);
  cudaError_t e = run_probe(out);
  return e == cudaSuccess ? FILTR_OK : cuda_fail(e, "probe");
}

}  // extern "C"
