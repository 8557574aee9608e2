// long.cu -- filtr_align_long: one long pair with every SM on it.
//
// X-drop pairs (and pairs with an empty side) run as a one-pair batch of the
// antidiagonal kernel with a 4-warp first window (reruns widen it); the
// antidiagonal order is inherently sequential, so one wide group is what the
// pair can use.  Full-matrix and banded pairs run the cooperative strip kernel
// (k_long.cu) across the whole grid, then the ordinary traceback walk.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/filtr_testing.h"
#include "filtr_ctx.h"
#include "k_strip.cuh"
#include "k_xdrop_layout.h"
#include "plan.h"

namespace filtr {

// X-drop pairs with more antidiagonals than this run as a segmented sweep, each
// segment at the narrowest group width that holds its live region
constexpr int64_t XD_SEGMENTED_SWEEP = 1 << 16;
namespace {

struct Carve {
  char *base;
  size_t cap, used = 0;
  template <class T>
  T *take(size_t count) {
    used = (used + 255) / 256 * 256;
    T *p = reinterpret_cast<T *>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

constexpr unsigned long long LONG_TIMEOUT_NS = 20ull * 1000 * 1000 * 1000;  // 20 s without progress

filtr_status validate_seq(Ctx *c, const uint8_t *q, uint32_t M, const uint8_t *r, uint32_t N,
                          int alphabet, cudaStream_t st) {
  uint32_t *d_bad = reinterpret_cast<uint32_t *>(c->d_small);
  cudaError_t e = cudaMemsetAsync(d_bad, 0, 4, st);
  if (e == cudaSuccess) e = launch_validate(q, M, alphabet, d_bad, st);
  if (e == cudaSuccess) e = launch_validate(r, N, alphabet, d_bad, st);
  if (!c->ensure_host(64)) return FILTR_ERR_NOMEM;
  uint32_t *h = reinterpret_cast<uint32_t *>(c->h_stage);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_bad, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "validating residues");
  if (*h) {
    set_error("%u residue codes are >= the alphabet size %d", *h, alphabet);
    return FILTR_ERR_INVALID;
  }
  return FILTR_OK;
}

// the cooperative strip kernel; withhold != 0 is the timeout test
filtr_status run_long(Ctx *c, const ScoreParams &sp, const filtr_params *params, const uint8_t *q,
                      uint32_t M, const uint8_t *r, uint32_t N, filtr_result *out, uint32_t *cigar,
                      uint64_t cap, cudaStream_t st, int withhold, unsigned long long timeout_ns,
                      bool sync = true) {
  constexpr int R = LONG_R, HS = 32 * R;
  int64_t lo = -(int64_t)M - 1, hi = (int64_t)N + 1;
  if (sp.use_band) {
    band_limits(M, N, sp.band, sp.band_literal, &lo, &hi);
    lo = std::max<int64_t>(lo, -(int64_t)M - 1);
    hi = std::min<int64_t>(hi, (int64_t)N + 1);
  }
  const int nstrips = (int)((M + HS - 1) / HS);
  // strip geometry: widest strip and traceback bases
  std::vector<int64_t> base(nstrips + 1, 0);
  int64_t widest = 0;
  for (int s = 0; s < nstrips; ++s) {
    int64_t jl, jh;
    strip_cols((int64_t)s * HS, HS, M, N, sp.use_band != 0, lo, hi, &jl, &jh);
    widest = std::max<int64_t>(widest, jh >= jl ? jh - jl + 1 : 0);
    base[s + 1] = base[s] + (sp.traceback ? strip_tb_words(jl, jh, R) : 0);
  }
  const uint64_t tb_words = (uint64_t)base[nstrips];
  const int bps = std::max(1, long_blocks_per_sm(sp));
  int grid = c->sms * bps;
  grid = std::max(1, std::min(grid, (nstrips + FULL_WARPS - 1) / FULL_WARPS));
  // the ring may use a quarter of the workspace
  const uint64_t stride = (uint64_t)widest + 2;
  while (grid > 1 && (uint64_t)grid * FULL_WARPS * stride * 8 > c->ws_bytes / 4) grid /= 2;
  if (withhold) grid = std::max(grid, 2);
  const int nw = grid * FULL_WARPS;

  Carve cv{c->ws, c->ws_bytes};
  int2 *ring = cv.take<int2>((size_t)nw * stride);
  unsigned long long *prog = cv.take<unsigned long long>(nw);
  int *err = cv.take<int>(4);
  LaneBest *wbest = cv.take<LaneBest>(nw);
  int *end_h = cv.take<int>(4);
  int64_t *d_base = cv.take<int64_t>(nstrips + 1);
  FwdOut *d_fwd = cv.take<FwdOut>(1);
  uint32_t *d_one = cv.take<uint32_t>(16);  // order, lengths, offsets of the one-pair batch
  TbLayout *d_tbl = cv.take<TbLayout>(1);
  uint64_t *d_misc = cv.take<uint64_t>(8);   // stage_off, offsets, total
  uint32_t *d_stage = sp.traceback ? cv.take<uint32_t>((size_t)M + N + 1) : nullptr;
  uint32_t *d_tb = cv.take<uint32_t>(tb_words);
  if (cv.used > c->ws_bytes) {
    set_error("the long pair needs %zu workspace bytes (traceback %llu); the context has %zu -- "
              "use a band, X-drop, or score only",
              cv.used, (unsigned long long)tb_words * 4, c->ws_bytes);
    return FILTR_ERR_NOMEM;
  }
  // host-side constants for the one-pair batch used by the walk
  if (!c->ensure_host(4096 + (nstrips + 1) * 8)) return FILTR_ERR_NOMEM;
  char *h = reinterpret_cast<char *>(c->h_stage);
  uint32_t one[16] = {0, M, N};            // order[0] = 0, q_len = M, r_len = N
  TbLayout L{};
  L.off = 0;
  L.family = FAM_FULL;
  L.R = R;
  L.warps = 1;
  L.valid = sp.traceback ? 1 : 0;
  uint64_t misc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // stage_off, q_off, r_off
  memcpy(h, one, sizeof one);
  memcpy(h + 64, &L, sizeof L);
  memcpy(h + 128, misc, sizeof misc);
  memcpy(h + 256, base.data(), (nstrips + 1) * 8);
  cudaError_t e = cudaMemcpyAsync(d_one, h, sizeof one, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tbl, h + 64, sizeof L, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_misc, h + 128, sizeof misc, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_base, h + 256, (nstrips + 1) * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(prog, 0, nw * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "long-pair setup");

  LongArgs a;
  a.q = q;
  a.r = r;
  a.M = (int)M;
  a.N = (int)N;
  a.lo = (int)lo;
  a.hi = (int)hi;
  a.sp = sp;
  a.ring = ring;
  a.ring_stride = (uint32_t)stride;
  a.prog = prog;
  a.err = err;
  a.timeout_ns = timeout_ns;
  a.withhold = withhold;
  a.tb = sp.traceback ? d_tb : nullptr;
  a.strip_base = d_base;
  a.wbest = wbest;
  a.end_h = end_h;
  c->span_begin(Ctx::PH_FORWARD, st);
  e = launch_long(a, grid, st);
  c->span_end(st);
  if (e != cudaSuccess) return cuda_fail(e, "long-pair kernel launch");
  const uint64_t cells = band_cells(M, N, sp);
  e = launch_long_finish(a, nw, cells, out, d_fwd, st);
  if (e != cudaSuccess) return cuda_fail(e, "long-pair finish");
  uint32_t launches = 2;
  if (sp.traceback && !withhold) {
    const uint64_t *d_off = d_misc + 1;
    BatchDev b{q, r, d_off, d_off + 1, d_one + 1, d_one + 2};
    WalkArgs wa;
    wa.b = b;
    wa.sp = sp;
    wa.order = d_one;
    wa.n_order = 1;
    wa.out = out;
    wa.fwd = d_fwd;
    wa.tb = d_tb;
    wa.tbl = d_tbl;
    wa.stage = d_stage;
    wa.stage_off = d_misc;
    c->span_begin(Ctx::PH_WALK, st);
    e = launch_walk(wa, st);
    c->span_end(st);
    if (e == cudaSuccess) e = launch_scan_offsets(out, 1, d_misc + 3, d_misc + 4, st);
    if (e == cudaSuccess) e = launch_compact(wa, 1, d_misc + 3, cigar, cap, out, st);
    launches += 3;
    if (e != cudaSuccess) return cuda_fail(e, "long-pair traceback");
  }
  c->last_launches = launches;
  c->last_cells_estimate = band_cells(M, N, sp);
  c->last_cells_packed = 0;
  c->last_waves = 1;
  if (!sync) return FILTR_OK;  // the result's status reports a timeout
  // the wait flag (and the CIGAR length) decide the status: synchronise once
  int *h_err = reinterpret_cast<int *>(h + 1024);
  filtr_result *h_res = reinterpret_cast<filtr_result *>(h + 1088);
  e = cudaMemcpyAsync(h_err, err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_res, out, sizeof(filtr_result), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "long-pair completion");
  if (*h_err) {
    set_error("a strip wait ran out after %llu ns", (unsigned long long)timeout_ns);
    return FILTR_ERR_TIMEOUT;
  }
  if (sp.traceback && h_res->cigar_len > cap) {
    set_error("the CIGAR needs %u ops, cigar_cap is %llu", h_res->cigar_len, (unsigned long long)cap);
    return FILTR_ERR_CIGAR_CAP;
  }
  return FILTR_OK;
}

// X-drop with checkpointed traceback (a one-pair antidiagonal sweep).
filtr_status run_xdrop_ckpt(Ctx *c, const ScoreParams &sp, const filtr_params *params,
                            const uint8_t *q, uint32_t M, const uint8_t *r, uint32_t N,
                            filtr_result *out, uint32_t *cigar, uint64_t cap, cudaStream_t st,
                            int C) {
  (void)params;
  const int64_t K = (int64_t)M + N;
  const int64_t nseg = (K + C - 1) / C;
  static const int kLadder[] = {1, 2, 4, 8, 16, XD_MAX_WARPS};
  Carve cv{c->ws, c->ws_bytes};
  int32_t *ck_buf = cv.take<int32_t>((size_t)(nseg + 1) * xd_ckpt_stride());
  const bool single = sp.traceback && !c->ckpt_recompute;
  uint32_t *seg_tb = (sp.traceback && !single)
                         ? cv.take<uint32_t>((size_t)C * xd_words_per_k(XD_MAX_WARPS, 8))
                         : nullptr;
  int32_t *seg_ck = (sp.traceback && !single) ? cv.take<int32_t>(C) : nullptr;
  XdCkpt *d_ck = cv.take<XdCkpt>(2 * nseg + 1);
  int32_t *d_flags = cv.take<int32_t>(nseg + 1);
  WalkState *d_ws = cv.take<WalkState>(1);
  FwdOut *d_fwd = cv.take<FwdOut>(1);
  uint32_t *d_one = cv.take<uint32_t>(16);   // order, lengths
  TbLayout *d_tbl = cv.take<TbLayout>(1);
  uint64_t *d_misc = cv.take<uint64_t>(8);   // stage_off, offsets, CIGAR offset
  uint32_t *d_ovf = cv.take<uint32_t>(4);
  uint32_t *d_stage = sp.traceback ? cv.take<uint32_t>((size_t)M + N + 1) : nullptr;
  // single pass: every segment's traceback rows kept in a pool (the rest of
  // the workspace), walked once at the end; if the pool runs out the sweep
  // stops and runs again without traceback, with the segments recomputed
  int32_t *seg_ck_all = single ? cv.take<int32_t>((size_t)nseg * C) : nullptr;
  uint64_t *seg_off = single ? cv.take<uint64_t>(nseg) : nullptr;
  int32_t *seg_wd = single ? cv.take<int32_t>(nseg) : nullptr;
  unsigned long long *pool_next = single ? cv.take<unsigned long long>(4) : nullptr;
  if (cv.used > c->ws_bytes) {
    set_error("checkpointed traceback needs %zu workspace bytes; the context has %zu", cv.used,
              c->ws_bytes);
    return FILTR_ERR_NOMEM;
  }
  uint32_t *pool = nullptr;
  uint64_t pool_words = 0;
  if (single) {
    pool = cv.take<uint32_t>(0);
    pool_words = cv.used < c->ws_bytes ? (c->ws_bytes - cv.used) / 4 : 0;
  }
  // host staging: the one-pair batch, the segment descriptors, the flags
  const size_t desc_off = 4096;
  const size_t flags_off = desc_off + (size_t)(2 * nseg + 1) * sizeof(XdCkpt);
  if (!c->ensure_host(flags_off + (size_t)(nseg + 1) * 4 + 64)) return FILTR_ERR_NOMEM;
  char *h = reinterpret_cast<char *>(c->h_stage);
  uint32_t one[16] = {0, M, N};  // order, q_len, r_len
  TbLayout L{};
  uint64_t misc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  memcpy(h, one, sizeof one);
  memcpy(h + 64, &L, sizeof L);
  memcpy(h + 128, misc, sizeof misc);
  XdCkpt *hk = reinterpret_cast<XdCkpt *>(h + desc_off);
  for (int64_t sgi = 0; sgi < nseg; ++sgi)
    hk[sgi] = XdCkpt{3,      C,          ck_buf,    (int)(sgi * C),
                     (int)std::min<int64_t>((sgi + 1) * C, K), nullptr, nullptr, d_flags,
                     pool,   pool_words, pool_next, seg_ck_all, seg_off, seg_wd};
  cudaError_t e = cudaMemcpyAsync(d_one, h, sizeof one, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && single) e = cudaMemsetAsync(pool_next, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tbl, h + 64, sizeof L, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_misc, h + 128, sizeof misc, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ck, hk, nseg * sizeof(XdCkpt), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_flags, 0, (nseg + 1) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ovf, 0, 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "checkpoint setup");
  const uint64_t *d_off = d_misc + 1;
  BatchDev b{q, r, d_off, d_off + 1, d_one + 1, d_one + 2};
  FullArgs fa;
  fa.b = b;
  fa.sp = sp;
  fa.sp.traceback = single ? 1 : 0;  // else the forward sweep keeps checkpoints only
  fa.order = d_one;
  fa.n_order = 1;
  fa.counter = nullptr;  // unused with checkpoints
  fa.out = out;
  fa.fwd = d_fwd;
  fa.tb = nullptr;
  fa.tbl = d_tbl;
  fa.strip_buf = nullptr;
  fa.strip_stride = 0;
  fa.max_n = 0;
  fa.max_m = 0;
  fa.x16_rebase = c->xd16_mode == 2 ? 0 : X16_REBASE;
  // forward: every segment is offered to each width in turn; the narrowest
  // window that holds it does the work, the other launches return at once
  uint32_t launches = 0;
  c->span_begin(Ctx::PH_FORWARD, st);
  for (int64_t sgi = 0; sgi < nseg && e == cudaSuccess; ++sgi) {
    fa.ck = d_ck + sgi;
    for (int W : kLadder) {
      e = launch_xdrop(fa, W, 1, d_ovf, d_ovf + 1, st);
      ++launches;
      if (e != cudaSuccess) break;
    }
  }
  c->span_end(st);
  FwdOut *hf = reinterpret_cast<FwdOut *>(h + 256);
  int32_t *hflags = reinterpret_cast<int32_t *>(h + flags_off);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, d_fwd, sizeof(FwdOut), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hflags, d_flags, (nseg + 1) * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "checkpointed forward sweep");
  const FwdOut f = *hf;
  c->last_launches = launches;
  if (hflags[0] == 3) {  // the packed sweep left its 16-bit range: the whole pair in int32
    ScoreParams s32 = sp;
    s32.xd16 = 0;
    const filtr_status rc = run_xdrop_ckpt(c, s32, params, q, M, r, N, out, cigar, cap, st, C);
    c->last_xd16 = 1;
    c->last_xd16_rerun = 1;
    return rc;
  }
  c->last_xd16 = sp.xd16 ? 1u : 0u;
  c->last_xd16_rerun = 0;
  if (single && hflags[0] == 2) {  // the pool ran out: recompute the segments instead
    const bool saved = c->ckpt_recompute;
    c->ckpt_recompute = true;
    const filtr_status rc = run_xdrop_ckpt(c, sp, params, q, M, r, N, out, cigar, cap, st, C);
    c->ckpt_recompute = saved;
    return rc;
  }
  if (!sp.traceback || (f.status != FILTR_ST_OK && f.status != FILTR_ST_DROPPED)) return FILTR_OK;
  WalkArgs wp;
  wp.b = b;
  wp.sp = sp;
  wp.order = d_one;
  wp.n_order = 1;
  wp.out = out;
  wp.fwd = d_fwd;
  wp.tb = nullptr;
  wp.tbl = d_tbl;
  wp.stage = d_stage;
  wp.stage_off = d_misc;
  if (single) {  // one walk over the kept traceback
    c->span_begin(Ctx::PH_WALK, st);
    e = launch_walk_pool(wp, pool, seg_ck_all, seg_off, seg_wd, C, st);
    c->span_end(st);
    uint64_t *d_offs = d_misc + 4;
    if (e == cudaSuccess) e = cudaMemsetAsync(d_offs, 0, 8, st);
    if (e == cudaSuccess) e = launch_compact(wp, 1, d_offs, cigar, cap, out, st);
    filtr_result *hr = reinterpret_cast<filtr_result *>(h + 1024);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr, out, sizeof(filtr_result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "single-pass traceback");
    c->last_launches = launches + 2;
    c->last_waves = 1;
    if (hr->cigar_len > cap) {
      set_error("the CIGAR needs %u ops, cigar_cap is %llu", hr->cigar_len, (unsigned long long)cap);
      return FILTR_ERR_CIGAR_CAP;
    }
    return FILTR_OK;
  }
  // backward: one segment at a time, from the end cell's antidiagonal down to
  // 0, each recomputed at the width that completed it going forward
  WalkState w0{f.end_i, f.end_j, f.score, 0, 0, -1, 0, 0};
  WalkState *hw = reinterpret_cast<WalkState *>(h + 512);
  *hw = w0;
  const int64_t ke = (int64_t)f.end_i + f.end_j;
  XdCkpt *hb = hk + nseg;
  std::vector<int> seg_w;
  int64_t nb = 0;
  for (int64_t khi = ke; khi > 0;) {
    const int64_t klo = ((khi - 1) / C) * C;
    const int W = hflags[1 + klo / C];
    if (W <= 0) {
      set_error("checkpointed sweep: segment at antidiagonal %lld has no width", (long long)klo);
      return FILTR_ERR_CUDA;
    }
    hb[nb++] = XdCkpt{2, C, ck_buf, (int)klo, (int)khi, seg_tb, seg_ck, d_flags};
    seg_w.push_back(W);
    khi = klo;
  }
  e = cudaMemcpyAsync(d_ws, hw, sizeof(WalkState), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nb)
    e = cudaMemcpyAsync(d_ck + nseg, hb, nb * sizeof(XdCkpt), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "segment setup");
  FullArgs ra = fa;
  ra.sp = sp;  // traceback on
  ra.out = reinterpret_cast<filtr_result *>(c->d_small + 3072);  // mode 2 writes no result
  WalkArgs wa;
  wa.b = b;
  wa.sp = sp;
  wa.order = d_one;
  wa.n_order = 1;
  wa.out = out;
  wa.fwd = d_fwd;
  wa.tb = nullptr;
  wa.tbl = d_tbl;
  wa.stage = d_stage;
  wa.stage_off = d_misc;
  for (int64_t sgi = 0; sgi < nb; ++sgi) {
    ra.ck = d_ck + nseg + sgi;
    e = launch_xdrop(ra, seg_w[sgi], 1, d_ovf, d_ovf + 1, st);
    if (e == cudaSuccess)
      e = launch_walk_segment(wa, seg_tb, seg_ck, hb[sgi].k_start, xd_words_per_k(seg_w[sgi], 8),
                              d_ws, st);
    launches += 2;
    if (e != cudaSuccess) return cuda_fail(e, "segment recompute");
  }
  uint64_t *d_offs = d_misc + 4;
  e = cudaMemsetAsync(d_offs, 0, 8, st);
  if (e == cudaSuccess) e = launch_compact(wa, 1, d_offs, cigar, cap, out, st);
  filtr_result *hr = reinterpret_cast<filtr_result *>(h + 1024);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hr, out, sizeof(filtr_result), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "checkpointed traceback");
  c->last_launches = launches + 1;
  c->last_waves = (int)nb;
  if (hr->cigar_len > cap) {
    set_error("the CIGAR needs %u ops, cigar_cap is %llu", hr->cigar_len, (unsigned long long)cap);
    return FILTR_ERR_CIGAR_CAP;
  }
  return FILTR_OK;
}

}  // namespace

// One long full-matrix / banded pair on the whole GPU without waiting for it
// (the serving loop's path for large requests).
filtr_status long_pair_async(Ctx *c, const ScoreParams &sp, const filtr_params *params,
                             const uint8_t *q, uint32_t M, const uint8_t *r, uint32_t N,
                             filtr_result *out, uint32_t *cigar, uint64_t cap, cudaStream_t st) {
  if (c->done_ev) cudaEventSynchronize(c->done_ev);
  c->ev_used = 0;
  c->spans.clear();
  const filtr_status rc =
      run_long(c, sp, params, q, M, r, N, out, cigar, cap, st, 0, LONG_TIMEOUT_NS, false);
  if (!c->done_ev) cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming);
  if (c->done_ev) cudaEventRecord(c->done_ev, st);
  return rc;
}

}  // namespace filtr

using namespace filtr;

extern "C" {

filtr_status filtr_align_long(filtr_ctx *ctx, const filtr_params *params, const uint8_t *q,
                              uint32_t M, const uint8_t *r, uint32_t N, filtr_result *out,
                              uint32_t *cigar, uint64_t cigar_cap, void *stream) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (sp.mid) {
    set_error("filtr_align_long: the M/I/D form runs only in filtr_align_batch");
    return FILTR_ERR_UNSUPPORTED;
  }
  if (!ctx || !out || (M && !q) || (N && !r) || (sp.traceback && cigar_cap && !cigar)) {
    set_error("filtr_align_long: NULL argument");
    return FILTR_ERR_INVALID;
  }
  if (M >= (1u << 30) || N >= (1u << 30)) {
    set_error("sequence longer than 2^30");
    return FILTR_ERR_UNSUPPORTED;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  if (c->done_ev) cudaEventSynchronize(c->done_ev);
  c->ev_used = 0;
  c->spans.clear();
  if (!score_range_ok(sp, M, N)) {
    set_error("scores could exceed 2^28 (2^26 for local alignments) for these lengths and penalties");
    return FILTR_ERR_UNSUPPORTED;
  }
  rc = validate_seq(c, q, M, r, N, sp.alphabet, st);
  if (rc != FILTR_OK) return rc;
  sp.xd16 = (c->xd16_mode != 1 && xd16_eligible(sp)) ? 1 : 0;
  if (sp.use_xdrop && M && N &&
      (c->ckpt_interval > 0 || (int64_t)M + N > XD_SEGMENTED_SWEEP ||
       4 * xd_tb_words(M, N, 32, 8) > c->ws_bytes / 2)) {  // the widest traceback would not fit
    const int C = c->ckpt_interval > 0 ? c->ckpt_interval : 4096;
    rc = run_xdrop_ckpt(c, sp, params, q, M, r, N, out, cigar, cigar_cap, st, C);
    if (!c->done_ev) cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming);
    if (c->done_ev) cudaEventRecord(c->done_ev, st);
    return rc;
  }
  if (sp.use_xdrop || M == 0 || N == 0 || (uint64_t)M * N < (1ull << 22) || M <= 512) {
    // a one-pair batch: lengths and offsets from the small device buffer
    uint64_t *d_off = reinterpret_cast<uint64_t *>(c->d_small + 1024);
    uint32_t *d_len = reinterpret_cast<uint32_t *>(c->d_small + 1088);
    if (!c->ensure_host(4096)) return FILTR_ERR_NOMEM;
    char *h = reinterpret_cast<char *>(c->h_stage);
    uint64_t offs[2] = {0, 0};
    uint32_t lens[2] = {M, N};
    memcpy(h + 2048, offs, sizeof offs);
    memcpy(h + 2112, lens, sizeof lens);
    cudaError_t e = cudaMemcpyAsync(d_off, h + 2048, sizeof offs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, h + 2112, sizeof lens, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the staging is reused by the batch call
    if (e != cudaSuccess) return cuda_fail(e, "one-pair setup");
    BatchDev b{q ? q : reinterpret_cast<const uint8_t *>(c->d_small),
               r ? r : reinterpret_cast<const uint8_t *>(c->d_small), d_off, d_off + 1, d_len, d_len + 1};
    const int w0 = c->xdrop_warps0;
    c->xdrop_warps0 = 4;
    rc = align_batch_impl(c, params, 1, b, out, cigar, cigar_cap, st, false, lens, lens + 1, true);
    c->xdrop_warps0 = w0;
    return rc;
  }
  rc = run_long(c, sp, params, q, M, r, N, out, cigar, cigar_cap, st, 0, LONG_TIMEOUT_NS);
  if (!c->done_ev) cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming);
  if (c->done_ev) cudaEventRecord(c->done_ev, st);
  return rc;
}

filtr_status filtr_test_set_checkpoint(filtr_ctx *ctx, int32_t interval) {
  if (!ctx || interval < 0) {
    set_error("filtr_test_set_checkpoint: bad arguments");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->ckpt_interval = interval;
  return FILTR_OK;
}

filtr_status filtr_test_set_first_width(filtr_ctx *ctx, int32_t warps) {
  if (!ctx || (warps != 0 && warps != 1 && warps != 2 && warps != 4 && warps != 8 && warps != 16 &&
               warps != 32)) {
    set_error("filtr_test_set_first_width: bad arguments");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->xdrop_warps0 = warps;
  return FILTR_OK;
}

filtr_status filtr_test_set_device_plan(filtr_ctx *ctx, int32_t mode) {
  if (!ctx || mode < 0 || mode > 2) {
    set_error("filtr_test_set_device_plan: bad arguments");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->dev_plan_mode = mode;
  return FILTR_OK;
}

filtr_status filtr_test_set_packed_sweep(filtr_ctx *ctx, int32_t mode) {
  if (!ctx || mode < 0 || mode > 2) {
    set_error("filtr_test_set_packed_sweep: bad arguments");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->xd16_mode = mode;
  return FILTR_OK;
}

filtr_status filtr_test_force_recompute(filtr_ctx *ctx, int32_t on) {
  if (!ctx) {
    set_error("filtr_test_force_recompute: ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->ckpt_recompute = on != 0;
  return FILTR_OK;
}

filtr_status filtr_test_long_timeout(filtr_ctx *ctx, const filtr_params *params, const uint8_t *q,
                                     uint32_t M, const uint8_t *r, uint32_t N,
                                     uint64_t timeout_ns) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (!ctx || !q || !r || M <= 512 || N == 0) {
    set_error("filtr_test_long_timeout: needs M > 512 and device sequences");
    return FILTR_ERR_INVALID;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaSetDevice(c->device);
  if (c->done_ev) cudaEventSynchronize(c->done_ev);
  sp.traceback = 0;
  filtr_result *d_out = reinterpret_cast<filtr_result *>(c->d_small + 2048);
  rc = run_long(c, sp, params, q, M, r, N, d_out, nullptr, 0, c->own_stream, 1, timeout_ns);
  return rc;
}

}  // extern "C"
