// filtr_internal.h -- shared definitions of the CUDA path (kernels + host code).
// Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/filtr.h"

#define FILTR_HD __host__ __device__ __forceinline__

namespace filtr {

// Logical minus infinity of the int32 kernels.  Finite scores stay far above
// NEG / 2 (|score| < 2^28 is enforced on the host), and a value produced from a
// NEG input stays far below NEG / 2, so "is it minus infinity" is x < NEG / 2.
constexpr int32_t NEG = -(1 << 29);
constexpr int32_t NEG_HALF = NEG / 2;
constexpr int MAX_ALPHA = 20;
constexpr int FULL_WARPS = 2;  // warps per CTA of the tiled wavefront kernel
// Rows per lane of the intra-pair strip kernel (strips of 32 * LONG_R rows).
// One long pair keeps only (strip width / strip height) strips in flight and
// each strip's step is latency bound, so lower strips (shorter steps, more of
// them in flight) finish sooner: an 80 kbp banded pair's forward took 48.2 ms
// at 8 rows against 55.1 ms at 16.
constexpr int LONG_R = 8;

// Band limits on d = j - i (Sec. 7.1 prune axis), widened to hold both corners
// unless the literal +-B band is asked for.
FILTR_HD void band_limits(int64_t M, int64_t N, int64_t B, bool literal, int64_t *lo,
                          int64_t *hi) {
  if (literal) {
    *lo = -B;
    *hi = B;
  } else {
    *lo = ((N - M) < 0 ? (N - M) : 0) - B;
    *hi = ((N - M) > 0 ? (N - M) : 0) + B;
  }
}

// Column range [jlo, jhi] (1-based) a row strip [row0 + 1, row0 + H] covers.
// Unbanded strips cover every column; banded ones only the band's columns.
FILTR_HD void strip_cols(int64_t row0, int64_t Hs, int64_t M, int64_t N, bool band, int64_t lo,
                         int64_t hi, int64_t *jlo, int64_t *jhi) {
  if (!band) {
    *jlo = 1;
    *jhi = N;
    return;
  }
  int64_t top = row0 + 1, bot = (row0 + Hs < M) ? row0 + Hs : M;
  int64_t a = top + lo, b = bot + hi;
  *jlo = a > 1 ? a : 1;
  *jhi = b < N ? b : N;
}

// Traceback words one strip of the tiled kernel writes: one step per column
// plus 31 pipeline steps, R/8 words per lane per step, 32 lanes.
FILTR_HD int64_t strip_tb_words(int64_t jlo, int64_t jhi, int R) {
  int64_t ncol = jhi >= jlo ? (jhi - jlo + 1) : 0;
  return ncol > 0 ? (ncol + 31) * (R / 8) * 32 : 0;
}

// Traceback bits.  Each cell contributes four bits, pushed most significant
// first into a 32-bit word by funnel shifts, so after 8 cells cell k sits in
// bits [4*(7-k), 4*(7-k)+4):
//   bit 3: E > D              (H came from E unless F wins)
//   bit 2: F > max(D, E)      (H came from F)
//   bit 1: E extended          (E_left - e > H_left - (o+e))
//   bit 0: F extended          (F_up - e > H_up - (o+e))
// Each bit is the sign of a difference (a - b < 0 <=> b > a); scores are below
// 2^30 in magnitude, so differences never overflow.
#ifdef __CUDACC__
__device__ __forceinline__ void tb_push4(uint32_t &w, int d3, int d2, int d1, int d0) {
  w = __funnelshift_l((uint32_t)d3, w, 1);
  w = __funnelshift_l((uint32_t)d2, w, 1);
  w = __funnelshift_l((uint32_t)d1, w, 1);
  w = __funnelshift_l((uint32_t)d0, w, 1);
}
#endif
enum : uint32_t { TB_PE = 8u, TB_PF = 4u, TB_EEXT = 2u, TB_FEXT = 1u };
FILTR_HD uint32_t tb_nibble(uint32_t word, int k) { return (word >> (4 * (7 - (k & 7)))) & 15u; }

// Per-pair output of the forward kernels before the traceback walk.
struct FwdOut {
  int32_t score;
  int32_t end_i, end_j;
  int32_t status;
};

// Kernel selection for one pair.
enum Family : uint8_t { FAM_FULL = 0, FAM_XDROP = 1, FAM_TRIVIAL = 2, FAM_PACK = 3 };

struct PairPlan {
  uint32_t pair;
  uint8_t family;
  uint8_t R;        // rows per lane (tiled kernel) or slots per lane (X-drop kernel)
  uint8_t warps;    // X-drop kernel: warps per CTA
  uint8_t pad;
  uint64_t tb_words;
  uint64_t cost;    // cell estimate for ordering
};

// What the traceback walk needs to find a cell's 4 bits.
struct TbLayout {
  uint64_t off;      // first word of this pair inside the traceback area
  uint8_t family;
  uint8_t R;
  uint8_t warps;
  uint8_t valid;     // 1 when this pair has traceback bits
  int32_t pad;
};

struct ScoreParams {
  int32_t mode, affine, o, e;  // o = 0 for linear gaps
  int32_t alphabet;
  int32_t use_band, band_literal, band;
  int32_t use_xdrop, xdrop;    // X-drop or Z-drop sweep, threshold
  int32_t zdrop;               // 1: Z-drop (distance from the best diagonal lowers the threshold)
  int32_t xrun;                // 1: threshold from the running best of all antidiagonals so far
  int32_t mid;                 // 1: Table 1's M/I/D form (gaps open from M), on the antidiagonal sweep
  int32_t traceback;
  int32_t precision;           // FILTR_PREC_*
  int32_t smin, smax;          // smallest / largest substitution score
  int32_t uni, uni_match, uni_mismatch;  // 1: one score on the diagonal, one off it
  int32_t xd16;                // 1: the antidiagonal sweep runs two cells per register
  int8_t subst[MAX_ALPHA * MAX_ALPHA];
};

// The packed (int16x2) antidiagonal sweep takes affine H/E/F pairs whose X-drop
// or Z-drop threshold leaves room in 15 bits around the running best; a pair
// whose values nevertheless leave the range stops with this internal status
// and is rerun by the int32 sweep.
constexpr int X16_MAX_DROP = 8000;
constexpr int X16_OVERFLOW = 64;
constexpr int X16_REBASE = 4096;  // distance of the best from the packed centre that moves the base
inline bool xd16_eligible(const ScoreParams &sp) {
  return sp.use_xdrop && sp.affine && !sp.mid && sp.xdrop < X16_MAX_DROP && sp.o + sp.e <= 1000 &&
         sp.smax <= 127 && sp.smin >= -128 && sp.precision != FILTR_PREC_I32;
}

// Score range of a batch whose longest query / reference are max_m / max_n:
// |H| stays below 2^28 so that NEG arithmetic never meets finite scores, and
// local scores stay below 2^26 so that the tiled kernels' best-cell keys
// (H * 32 + row) fit in 31 bits.
inline bool score_range_ok(const ScoreParams &sp, uint64_t max_m, uint64_t max_n) {
  int smax = 0;
  for (int t = 0; t < sp.alphabet * sp.alphabet; ++t) {
    const int v = sp.subst[t] < 0 ? -sp.subst[t] : sp.subst[t];
    smax = v > smax ? v : smax;
  }
  const double shorter = (double)(max_m < max_n ? max_m : max_n);
  const double bound = (double)smax * shorter + 3.0 * (double)sp.o +
                       (double)sp.e * (double)(max_m + max_n);
  if (bound >= (double)(1 << 28)) return false;
  return sp.mode != FILTR_LOCAL || (double)smax * shorter < (double)(1 << 26);
}

// ---- packed 16-bit cells (two per 32-bit register) ---------------------------
// A value v is held as the unsigned 16-bit v + B.  B is chosen per pair so that
// every quantity the recurrence forms (H, E, F, the diagonal candidate and the
// gap candidates) lies in [0, 0x8000): then sums never carry or borrow across
// the halves, unsigned max is signed max, and A - B + 0x7fff leaves [A > B] in
// bit 15 of each half.  Returns B, or -1 when the pair's bound does not fit
// (the pair then runs in int32).  Unbanded alignments only; substitution
// scores must lie in [-64, 63] (the profile holds s + 64 in 7 bits).
FILTR_HD int pack_bias(int mode, int o, int e, int smin, int smax, int64_t M, int64_t N) {
  if (smin < -64 || smax > 63) return -1;
  const int64_t oe = (int64_t)o + e;
  // lowest value any formed quantity can take:
  //   local:  H >= 0, E, F >= -(o+e), extensions a further -e, diagonal >= smin
  //   global: H(i,j) >= -(2o + e(i+j)) (a gap down the first column, then one
  //           along row i), then the same offsets
  int64_t low = oe + e + 64;
  if (mode != FILTR_LOCAL) low += 2 * (int64_t)o + (int64_t)e * (M + N);
  const int64_t B = low + e + 2;
  const int64_t high = (int64_t)(smax > 0 ? smax : 0) * ((M < N ? M : N) + 1) + 2;
  if (B + high >= 0x7ff0) return -1;
  return (int)B;
}
// Packed tile: words per lane and step -- each half's R/2 cells fill
// ceil(R/16) words of four 8-cell bit planes.
FILTR_HD int pack_words_per_step(int R) { return 2 * ((R / 2 + 7) / 8); }
// Packed tile query profile: per residue, 32 lanes x two halves x ceil(R/8)
// words (each half's R/2 bytes padded to whole words).
FILTR_HD constexpr int pack_prof_stride(int R) { return 256 * ((R / 2 + 3) / 4); }
FILTR_HD uint64_t pack_strip_tb_words(int64_t jlo, int64_t jhi, int R) {
  return jhi >= jlo ? (uint64_t)((jhi - jlo + 1) + 63) * (uint64_t)pack_words_per_step(R) * 32u : 0;
}

struct BatchDev {
  const uint8_t *q_seq, *r_seq;
  const uint64_t *q_off, *r_off;
  const uint32_t *q_len, *r_len;
};

// Per-launch values of a captured batch pipeline (filtr_graph), in device
// memory.  A graph's kernels are captured once with fixed by-value arguments;
// where a kernel's gd argument is set it takes the batch, the pair count and
// the outputs from here instead (written by the graph's first node at each
// launch), and does nothing once abort is set (a check node found a residue
// code or a length outside the graph's bounds, or traceback over its budget).
struct GraphDesc {
  BatchDev b;
  filtr_result *out;
  uint32_t *cigar;
  uint64_t cap;
  uint32_t n;
  int32_t abort;   // 0, or the filtr_status that stopped this launch
};
struct DevPlanSummary;

struct FullArgs {
  BatchDev b;
  ScoreParams sp;
  const uint32_t *order;   // pairs this launch handles, in processing order
  uint32_t n_order;
  uint32_t *counter;       // work-queue cursor (zeroed before launch)
  filtr_result *out;
  FwdOut *fwd;             // per pair (indexed by pair id)
  uint32_t *tb;            // traceback area
  const TbLayout *tbl;     // per pair
  int2 *strip_buf;         // per resident warp: strip_stride entries
  uint32_t strip_stride;
  uint32_t max_n;          // 0, or the longest reference the strip buffers hold
  uint32_t max_m;          // 0, or the longest query accepted
  const struct XdCkpt *ck; // X-drop kernel: checkpoint mode (nullptr = normal)
  // packed X-drop sweep: pairs that left the 16-bit range (rerun in int32),
  // and the base move distance (<= 0: never, a test hook)
  uint32_t *ovf16 = nullptr;
  uint32_t *n_ovf16 = nullptr;
  int x16_rebase = X16_REBASE;
  // captured pipeline (tiled kernels only): b and out come from gd, and the
  // launch takes order[begin, begin + count[gshape]) with begin the pairs of
  // the shapes before gshape in the device plan's summary
  const GraphDesc *gd = nullptr;
  const DevPlanSummary *gsum = nullptr;
  int gshape = 0;
};

struct WalkArgs {
  BatchDev b;
  ScoreParams sp;
  const uint32_t *order;
  uint32_t n_order;
  filtr_result *out;
  const FwdOut *fwd;
  const uint32_t *tb;
  const TbLayout *tbl;
  uint32_t *stage;          // per pair scratch for reversed CIGAR ops
  const uint64_t *stage_off;
  const GraphDesc *gd = nullptr;  // captured pipeline: b, out and n_order from here
};

struct LaneBest;
// One long pair across the whole grid (k_long.cu).
struct LongArgs {
  const uint8_t *q, *r;
  int M, N;
  int lo, hi;                 // band on j - i (unbanded: -M-1, N+1)
  ScoreParams sp;
  int2 *ring;                 // NW slots of ring_stride entries
  uint32_t ring_stride;
  unsigned long long *prog;   // NW progress words (strip << 32 | column), zeroed
  int *err;                   // set to 1 when a wait times out
  unsigned long long timeout_ns;
  int withhold;               // test hook: strip 0 never publishes (forces the timeout)
  uint32_t *tb;               // traceback words (nullptr without traceback)
  const int64_t *strip_base;  // first traceback word of each strip
  struct LaneBest *wbest;     // one per warp
  int *end_h;                 // H(M, N)
};

// ---- launches (defined in the .cu files) -----------------------------------
cudaError_t launch_long(const LongArgs &a, int grid, cudaStream_t s);
cudaError_t launch_long_finish(const LongArgs &a, int nw, uint64_t cells, filtr_result *out,
                               FwdOut *fwd, cudaStream_t s);
int long_blocks_per_sm(const ScoreParams &sp);
cudaError_t launch_full(const FullArgs &a, int R, int grid, cudaStream_t s);
int full_smem_bytes(int R, int alphabet);
int full_max_blocks_per_sm(int R, const ScoreParams &sp, int alphabet);
// int16x2 tile, every even R from 8 to 32 (k_pack.cu dispatches; instances in
// k_pack.cu, k_pack_mid.cu, k_pack_odd.cu and k_pack_odd_hi.cu)
cudaError_t launch_pack(const FullArgs &a, int R, int grid, cudaStream_t s);
int pack_max_blocks_per_sm(int R, const ScoreParams &sp);
cudaError_t launch_pack_mid(const FullArgs &a, int R, int grid, cudaStream_t s);
int pack_mid_blocks_per_sm(int R, const ScoreParams &sp);
cudaError_t launch_pack_odd(const FullArgs &a, int R, int grid, cudaStream_t s);  // R = 10, ..., 30
int pack_odd_blocks_per_sm(int R, const ScoreParams &sp);
// occupancy of the captured-pipeline instances (launch_full / launch_pack pick
// them when FullArgs::gd is set)
int full_graph_blocks_per_sm(int R, const ScoreParams &sp);
int pack_graph_blocks_per_sm(int R, const ScoreParams &sp);
inline int pack_smem_bytes(int R, int alphabet) {
  return 512 + FULL_WARPS * alphabet * pack_prof_stride(R);
}
cudaError_t launch_xdrop(const FullArgs &a, int W, int grid, uint32_t *overflow,
                         uint32_t *n_overflow, cudaStream_t s);
int xd_pairs_per_cta(int W, const ScoreParams &sp);
struct WalkState;
cudaError_t launch_walk_segment(const WalkArgs &a, const uint32_t *seg_tb, const int32_t *seg_ck,
                                int k_start, int wpk, WalkState *st, cudaStream_t s);
int xd_max_blocks_per_sm(int W, const ScoreParams &sp);
cudaError_t launch_walk(const WalkArgs &a, cudaStream_t s);
cudaError_t launch_walk_xd(const WalkArgs &a, cudaStream_t s);  // X-drop pairs, a warp each
cudaError_t launch_walk_pool(const WalkArgs &a, const uint32_t *pool, const int32_t *seg_ck_all,
                             const uint64_t *seg_off, const int32_t *seg_w, int C, cudaStream_t s);
// In a captured pipeline (gd set) the n given here is the graph's capacity,
// which sizes the grid; the kernels take the launch's n from gd.
cudaError_t launch_scan_offsets(const filtr_result *out, uint32_t n, uint64_t *offs,
                                uint64_t *total, cudaStream_t s, const GraphDesc *gd = nullptr);
cudaError_t launch_compact(const WalkArgs &a, uint32_t n, const uint64_t *offs, uint32_t *cigar,
                           uint64_t cap, filtr_result *out, cudaStream_t s);
cudaError_t launch_trivial(const BatchDev &b, const ScoreParams &sp, const uint32_t *order,
                           uint32_t n, filtr_result *out, FwdOut *fwd, cudaStream_t s,
                           const GraphDesc *gd = nullptr, const DevPlanSummary *gsum = nullptr);
cudaError_t launch_validate(const uint8_t *codes, uint64_t n, int alphabet, uint32_t *bad,
                            cudaStream_t s);
cudaError_t launch_validate_pairs(const BatchDev &b, uint32_t n, int alphabet, uint32_t *bad,
                                  cudaStream_t s, const GraphDesc *gd = nullptr);
cudaError_t launch_pack(const uint8_t *codes, uint64_t n, int alphabet, uint32_t *packed,
                        uint32_t *bad, cudaStream_t s);
cudaError_t run_probe(double out[5]);

// ---- host-side error reporting ---------------------------------------------
void set_error(const char *fmt, ...);
filtr_status cuda_fail(cudaError_t e, const char *what);

}  // namespace filtr
