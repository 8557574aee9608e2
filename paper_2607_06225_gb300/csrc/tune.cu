// tune.cu -- filtr_autotune: measured costs of the tiled kernel shapes.
//
// The planner gives each pair the tiled shape (the int32 tile with R = 32, 24,
// 16 or 8 rows per lane, or the int16x2 tile with R = 32, 28, ..., 8) whose predicted
// time, strips x (N + fill steps) x cost-per-warp-step, is smallest.  The
// built-in costs come from instruction counts; this entry point replaces them
// with the device time per warp step measured on this GPU for one recurrence
// kind: each shape runs a batch that fills every resident warp slot three
// times over with pairs of one full strip (32R query rows) by 512 reference
// residues of random codes, and the cost is the launch's duration divided by
// the warp steps it executed.  Shapes are bit-exact alternatives, so tuning
// changes speed only.
//
// With X-drop / Z-drop parameters it tunes the antidiagonal sweep instead: the
// int16x2 and int32 sweeps at a first group width of 1 and 2 (256 and 512 slots) each run
// a batch of related pairs (2048-residue random references, queries with 5%
// substitutions, 2% insertions and 2% deletions) that fills the device twice,
// and the context keeps the width and cell width with the smallest time per
// evaluated cell among those that finished nearly every pair without
// outgrowing their window.
#include <algorithm>
#include <cstring>
#include <vector>

#include "filtr_ctx.h"
#include "k_xdrop_layout.h"

namespace filtr {
namespace {

constexpr int TUNE_N = 512;
constexpr int TUNE_ROUNDS = 3;

struct TuneCarve {
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

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Time one shape; returns ns per warp step, or a negative value if the
// workspace cannot hold a batch that fills the device once.
double time_shape(Ctx *c, const ScoreParams &sp, const ShapeCost &shape, cudaStream_t st,
                  filtr_status *rc) {
  *rc = FILTR_OK;
  const int R = shape.R, M = 32 * R, N = TUNE_N;
  const int bps = shape.packed ? c->pack_blocks_per_sm(R, sp) : c->full_blocks_per_sm(R, sp);
  const int grid = c->sms * bps;
  const int64_t slots = (int64_t)grid * FULL_WARPS;
  uint64_t tbw = 0;
  if (sp.traceback)
    tbw = shape.packed ? pack_strip_tb_words(1, N, R) : full_tb_words(M, N, R, sp);
  auto bytes_for = [&](int64_t B) {
    return (size_t)B * (M + N) + (size_t)B * (16 + 8 + sizeof(filtr_result) + sizeof(FwdOut) +
                                              sizeof(TbLayout)) +
           (size_t)slots * (N + 2) * sizeof(int2) + (size_t)B * tbw * 4 + 64 * 256;
  };
  int64_t B = slots * TUNE_ROUNDS;
  while (B > slots && bytes_for(B) > c->ws_bytes) B -= slots;
  if (bytes_for(B) > c->ws_bytes) return -1.0;

  TuneCarve cv{c->ws, c->ws_bytes};
  uint8_t *d_codes = cv.take<uint8_t>((size_t)B * (M + N));
  uint64_t *d_off = cv.take<uint64_t>(2 * B);
  uint32_t *d_len = cv.take<uint32_t>(2 * B);
  filtr_result *d_out = cv.take<filtr_result>(B);
  FwdOut *d_fwd = cv.take<FwdOut>(B);
  TbLayout *d_tbl = cv.take<TbLayout>(B);
  uint32_t *d_counter = cv.take<uint32_t>(64);
  int2 *d_strip = cv.take<int2>((size_t)slots * (N + 2));
  uint32_t *d_tb = sp.traceback ? cv.take<uint32_t>((size_t)B * tbw) : nullptr;

  // random codes, offsets (queries first, then references), lengths, layouts
  std::vector<uint8_t> codes((size_t)B * (M + N));
  uint64_t seed = 0x5eed0001ull + (uint64_t)R * 131 + (shape.packed ? 7 : 0);
  for (size_t i = 0; i < codes.size(); i += 8) {
    uint64_t v = splitmix(seed);
    for (size_t b = 0; b < 8 && i + b < codes.size(); ++b)
      codes[i + b] = (uint8_t)(((v >> (8 * b)) & 0xffu) % (uint64_t)sp.alphabet);
  }
  std::vector<uint64_t> offs(2 * B);
  std::vector<uint32_t> lens(2 * B);
  std::vector<TbLayout> tbl(B);
  for (int64_t p = 0; p < B; ++p) {
    offs[p] = (uint64_t)p * M;
    offs[B + p] = (uint64_t)B * M + (uint64_t)p * N;
    lens[p] = (uint32_t)M;
    lens[B + p] = (uint32_t)N;
    tbl[p] = TbLayout{};
    tbl[p].off = (uint64_t)p * tbw;
    tbl[p].family = shape.packed ? FAM_PACK : FAM_FULL;
    tbl[p].R = (uint8_t)R;
    tbl[p].warps = 1;
    tbl[p].valid = sp.traceback ? 1 : 0;
  }
  cudaError_t e = cudaMemcpyAsync(d_codes, codes.data(), codes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_len, lens.data(), lens.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tbl, tbl.data(), tbl.size() * sizeof(TbLayout), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "autotune upload");
    return -1.0;
  }
  FullArgs fa{};
  fa.b = BatchDev{d_codes, d_codes, d_off, d_off + B, d_len, d_len + B};
  fa.sp = sp;
  fa.order = nullptr;
  fa.n_order = (uint32_t)B;
  fa.out = d_out;
  fa.fwd = d_fwd;
  fa.tb = d_tb;
  fa.tbl = d_tbl;
  fa.strip_buf = d_strip;
  fa.strip_stride = N + 2;
  fa.max_n = 0;
  fa.max_m = 0;
  fa.ck = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = -1.0f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // one warm-up, two timed
    fa.counter = d_counter + 4 * rep;
    e = cudaMemsetAsync(fa.counter, 0, 4, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess)
      e = shape.packed ? launch_pack(fa, R, grid, st) : launch_full(fa, R, grid, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best_ms < 0 || ms < best_ms)) best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "autotune launch");
    return -1.0;
  }
  const double warp_steps = (double)B * (double)(N + shape.fill);
  return (double)best_ms * 1e6 / warp_steps;
}

constexpr int SWEEP_L = 2048;
// the sweep candidates, in the order filtr_autotune reports them: (warps, packed)
constexpr int SWEEP_CAND = 4;
constexpr int kSweepW[SWEEP_CAND] = {1, 1, 2, 2};
constexpr int kSweepPacked[SWEEP_CAND] = {1, 0, 1, 0};

// Time one sweep candidate; returns ns per evaluated cell of the pairs that
// finished, or a negative value when it cannot run here (workspace too small,
// not eligible, or more than 1% of the pairs outgrew the window).
double time_sweep(Ctx *c, const ScoreParams &sp0, int W, bool packed, cudaStream_t st,
                  filtr_status *rc) {
  *rc = FILTR_OK;
  ScoreParams sp = sp0;
  sp.xd16 = packed ? 1 : 0;
  if (packed && !xd16_eligible(sp0)) return -1.0;
  const int ppc = xd_pairs_per_cta(W, sp);
  const int bps = std::max(1, xd_max_blocks_per_sm(W, sp));
  const int grid = c->sms * bps;
  // the reference and the query of every pair, generated once on the host
  std::vector<uint8_t> ref, qry;
  std::vector<uint32_t> qlen;
  int64_t B = (int64_t)grid * ppc * 2;
  const uint64_t tbw = sp.traceback ? xd_tb_words(SWEEP_L + SWEEP_L / 16, SWEEP_L, W, 8) : 0;
  auto bytes_for = [&](int64_t n) {
    return (size_t)n * (2 * SWEEP_L + SWEEP_L / 8) +
           (size_t)n * (16 + 8 + sizeof(filtr_result) + sizeof(FwdOut) + sizeof(TbLayout) + 4) +
           (size_t)n * tbw * 4 + 64 * 256;
  };
  while (B > grid && bytes_for(B) > c->ws_bytes) B -= grid;
  if (bytes_for(B) > c->ws_bytes) return -1.0;
  uint64_t seed = 0x5eed1000ull + (uint64_t)W * 17 + (packed ? 3 : 0);
  const int A = sp.alphabet;
  ref.resize((size_t)B * SWEEP_L);
  for (auto &x : ref) x = (uint8_t)(splitmix(seed) % (uint64_t)A);
  qlen.resize(B);
  for (int64_t p = 0; p < B; ++p) {
    const uint8_t *r = ref.data() + (size_t)p * SWEEP_L;
    const size_t q0 = qry.size();
    // queries stop at SWEEP_L + SWEEP_L / 16 residues, the length the
    // traceback areas are sized for
    for (int j = 0; j < SWEEP_L && qry.size() - q0 + 2 <= (size_t)(SWEEP_L + SWEEP_L / 16); ++j) {
      const uint64_t u = splitmix(seed) % 100;
      if (u < 5) {
        qry.push_back((uint8_t)((r[j] + 1 + splitmix(seed) % (uint64_t)(A - 1)) % (uint64_t)A));
      } else if (u < 7) {
        qry.push_back((uint8_t)(splitmix(seed) % (uint64_t)A));
        qry.push_back(r[j]);
      } else if (u >= 9) {
        qry.push_back(r[j]);
      }  // 7 <= u < 9: deleted
    }
    qlen[p] = (uint32_t)(qry.size() - q0);
  }
  TuneCarve cv{c->ws, c->ws_bytes};
  uint8_t *d_codes = cv.take<uint8_t>(ref.size() + qry.size());
  uint64_t *d_off = cv.take<uint64_t>(2 * B);
  uint32_t *d_len = cv.take<uint32_t>(2 * B);
  filtr_result *d_out = cv.take<filtr_result>(B);
  FwdOut *d_fwd = cv.take<FwdOut>(B);
  TbLayout *d_tbl = cv.take<TbLayout>(B);
  uint32_t *d_order = cv.take<uint32_t>(B);
  uint32_t *d_counter = cv.take<uint32_t>(64);
  uint32_t *d_ovf = cv.take<uint32_t>(B);
  uint32_t *d_ovf16 = cv.take<uint32_t>(B);
  uint32_t *d_novf = cv.take<uint32_t>(8);
  uint32_t *d_tb = sp.traceback ? cv.take<uint32_t>((size_t)B * tbw) : nullptr;
  if (cv.used > c->ws_bytes) return -1.0;
  std::vector<uint64_t> offs(2 * B);
  std::vector<uint32_t> lens(2 * B), order(B);
  std::vector<TbLayout> tbl(B);
  uint64_t qo = 0;
  for (int64_t p = 0; p < B; ++p) {
    offs[p] = qo;
    qo += qlen[p];
    offs[B + p] = qry.size() + (uint64_t)p * SWEEP_L;
    lens[p] = qlen[p];
    lens[B + p] = SWEEP_L;
    order[p] = (uint32_t)p;
    tbl[p] = TbLayout{};
    tbl[p].off = (uint64_t)p * tbw;
    tbl[p].family = FAM_XDROP;
    tbl[p].R = 8;
    tbl[p].warps = (uint8_t)W;
    tbl[p].valid = sp.traceback ? 1 : 0;
  }
  cudaError_t e = cudaMemcpyAsync(d_codes, qry.data(), qry.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_codes + qry.size(), ref.data(), ref.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, lens.data(), lens.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tbl, tbl.data(), tbl.size() * sizeof(TbLayout), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "autotune upload");
    return -1.0;
  }
  FullArgs fa{};
  fa.b = BatchDev{d_codes, d_codes, d_off, d_off + B, d_len, d_len + B};
  fa.sp = sp;
  fa.order = d_order;
  fa.n_order = (uint32_t)B;
  fa.out = d_out;
  fa.fwd = d_fwd;
  fa.tb = d_tb;
  fa.tbl = d_tbl;
  fa.ck = nullptr;
  fa.ovf16 = d_ovf16;
  fa.n_ovf16 = d_novf + 4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = -1.0f;
  const int gl = (int)std::min<int64_t>((int64_t)grid, (B + ppc - 1) / ppc);
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // one warm-up, two timed
    fa.counter = d_counter + 4 * rep;
    e = cudaMemsetAsync(fa.counter, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_novf, 0, 32, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_xdrop(fa, W, std::max(gl, 1), d_ovf, d_novf, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best_ms < 0 || ms < best_ms)) best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<filtr_result> res(B);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res.data(), d_out, B * sizeof(filtr_result), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "autotune launch");
    return -1.0;
  }
  uint64_t cells = 0;
  int64_t unfinished = 0;
  for (const filtr_result &r : res) {
    if (r.status == FILTR_ST_TOO_WIDE) ++unfinished;
    else cells += r.cells;
  }
  if (unfinished * 100 > B || cells == 0) return -1.0;
  return (double)best_ms * 1e6 / (double)cells;
}

// Keep measured costs (ns per warp step; 0 = not timed) for this recurrence
// kind.  Untimed shapes keep the model's cost scaled to the timed ones.
void install_costs(Ctx *c, const ScoreParams &sp, const double *ns_k) {
  std::vector<ShapeCost> tab(kDefaultShapeCost, kDefaultShapeCost + SHAPE_TILED);
  double scale_num = 0, scale_den = 0;
  for (int k = 0; k < SHAPE_TILED; ++k)
    if (ns_k[k] > 0) {
      const ShapeCost &d = kDefaultShapeCost[k];
      scale_num += ns_k[k];
      scale_den += d.per_row * d.R + d.per_step;
    }
  for (int k = 0; k < SHAPE_TILED; ++k) {
    const double model = tab[k].per_row * tab[k].R + tab[k].per_step;
    tab[k].per_row = 0.0f;
    tab[k].per_step = (float)(ns_k[k] > 0 ? ns_k[k]
                                          : (scale_den > 0 ? model * scale_num / scale_den : model));
  }
  c->tuned[Ctx::tune_key(sp)] = tab;
}

}  // namespace
}  // namespace filtr

using namespace filtr;

extern "C" filtr_status filtr_autotune(filtr_ctx *ctx, const filtr_params *params,
                                       filtr_tune_report *out) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (!ctx) {
    set_error("filtr_autotune: ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (c->done_ev) {
    e = cudaEventSynchronize(c->done_ev);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the previous call");
  }
  cudaStream_t st = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  static_assert(SHAPE_TILED <= FILTR_TUNE_MAX_SHAPES, "tune report too small");
  if (sp.use_xdrop) {  // the antidiagonal sweep: cell width and first group width
    if (out) {
      memset(out, 0, sizeof *out);
      out->n_shapes = SWEEP_CAND;
    }
    int bestk = -1;
    double bestns = 0;
    for (int k = 0; k < SWEEP_CAND; ++k) {
      if (out) {
        out->rows_per_lane[k] = kSweepW[k];
        out->packed[k] = kSweepPacked[k];
      }
      if (kSweepPacked[k] && (sp.mid || sp.precision == FILTR_PREC_I32)) continue;
      filtr_status trc = FILTR_OK;
      const double ns = time_sweep(c, sp, kSweepW[k], kSweepPacked[k] != 0, st, &trc);
      if (trc != FILTR_OK) {
        cudaStreamDestroy(st);
        return trc;
      }
      if (ns <= 0) continue;
      if (out) out->ns_per_warp_step[k] = ns;
      if (bestk < 0 || ns < bestns) {
        bestk = k;
        bestns = ns;
      }
    }
    cudaStreamDestroy(st);
    if (bestk < 0) {
      set_error("filtr_autotune: no sweep candidate ran (workspace too small, or every width too narrow)");
      return FILTR_ERR_NOMEM;
    }
    c->sweep_tuned[Ctx::sweep_key(sp)] = Ctx::SweepChoice{kSweepPacked[bestk], kSweepW[bestk]};
    return FILTR_OK;
  }
  if (out) {
    memset(out, 0, sizeof *out);
    out->n_shapes = SHAPE_TILED;
  }
  double ns_k[SHAPE_TILED] = {};
  bool any = false;
  for (int k = 0; k < SHAPE_TILED; ++k) {
    const ShapeCost &s = kDefaultShapeCost[k];
    if (out) {
      out->rows_per_lane[k] = s.R;
      out->packed[k] = s.packed ? 1 : 0;
    }
    const bool can_pack = !sp.use_band && sp.precision != FILTR_PREC_I32 &&
                          pack_bias(sp.mode, sp.o, sp.e, sp.smin, sp.smax, 32 * s.R, TUNE_N) >= 0;
    if (s.packed && !can_pack) continue;  // the planner never picks it for this kind
    filtr_status trc = FILTR_OK;
    const double ns = time_shape(c, sp, s, st, &trc);
    if (trc != FILTR_OK) {
      cudaStreamDestroy(st);
      return trc;
    }
    if (ns <= 0) continue;  // keeps the built-in estimate
    ns_k[k] = ns;
    any = true;
    if (out) out->ns_per_warp_step[k] = ns;
  }
  cudaStreamDestroy(st);
  if (!any) {
    set_error("filtr_autotune: the workspace cannot hold one calibration batch");
    return FILTR_ERR_NOMEM;
  }
  install_costs(c, sp, ns_k);
  return FILTR_OK;
}

extern "C" filtr_status filtr_tune_apply(filtr_ctx *ctx, const filtr_params *params,
                                         const filtr_tune_report *report) {
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (!ctx || !report) {
    set_error("filtr_tune_apply: ctx or report is NULL");
    return FILTR_ERR_INVALID;
  }
  if (sp.use_xdrop) {  // a sweep report: the fastest timed candidate
    if (report->n_shapes != SWEEP_CAND) {
      set_error("filtr_tune_apply: an X-drop report lists %d sweep candidates, not %d", report->n_shapes,
                SWEEP_CAND);
      return FILTR_ERR_INVALID;
    }
    int bestk = -1;
    for (int k = 0; k < SWEEP_CAND; ++k) {
      if (report->rows_per_lane[k] != kSweepW[k] || report->packed[k] != kSweepPacked[k]) {
        set_error("filtr_tune_apply: sweep candidate %d is not (warps=%d, packed=%d)", k, kSweepW[k],
                  kSweepPacked[k]);
        return FILTR_ERR_INVALID;
      }
      const double ns = report->ns_per_warp_step[k];
      if (!(ns >= 0.0 && ns < 1e9)) {
        set_error("filtr_tune_apply: ns_per_warp_step[%d] must be finite and >= 0", k);
        return FILTR_ERR_INVALID;
      }
      if (ns > 0 && (bestk < 0 || ns < report->ns_per_warp_step[bestk])) bestk = k;
    }
    if (bestk < 0) {
      set_error("filtr_tune_apply: the report holds no timed candidate");
      return FILTR_ERR_INVALID;
    }
    reinterpret_cast<Ctx *>(ctx)->sweep_tuned[Ctx::sweep_key(sp)] =
        Ctx::SweepChoice{kSweepPacked[bestk], kSweepW[bestk]};
    return FILTR_OK;
  }
  double ns_k[SHAPE_TILED] = {};
  bool any = false;
  if (report->n_shapes != SHAPE_TILED) {
    set_error("filtr_tune_apply: the report lists %d shapes, this library has %d", report->n_shapes,
              SHAPE_TILED);
    return FILTR_ERR_INVALID;
  }
  for (int k = 0; k < SHAPE_TILED; ++k) {
    const ShapeCost &d = kDefaultShapeCost[k];
    if (report->rows_per_lane[k] != d.R || report->packed[k] != (d.packed ? 1 : 0)) {
      set_error("filtr_tune_apply: shape %d is not (R=%d, packed=%d) as filtr_autotune reports it",
                k, d.R, d.packed ? 1 : 0);
      return FILTR_ERR_INVALID;
    }
    const double ns = report->ns_per_warp_step[k];
    if (!(ns >= 0.0 && ns < 1e9)) {  // also rejects NaN
      set_error("filtr_tune_apply: ns_per_warp_step[%d] must be finite and >= 0", k);
      return FILTR_ERR_INVALID;
    }
    ns_k[k] = ns;
    any = any || ns > 0;
  }
  if (!any) {
    set_error("filtr_tune_apply: the report holds no timed shape");
    return FILTR_ERR_INVALID;
  }
  install_costs(reinterpret_cast<Ctx *>(ctx), sp, ns_k);
  return FILTR_OK;
}
