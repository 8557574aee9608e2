// k_xdrop_layout.h -- traceback layout of the antidiagonal (X-drop) kernel.
//
// Per pair: (M + N + 1) int32 window origins c_k (the column j of slot 0 on
// antidiagonal k), padded to a multiple of 8 words, then for every antidiagonal
// k a window of WPK words holding one 4-bit nibble per slot (slot p <-> cell
// (k - c_k - p, c_k + p)).
#pragma once

#include "filtr_internal.h"

namespace filtr {

FILTR_HD int xd_window_slots(int warps, int S) { return warps * 32 * S; }
FILTR_HD int xd_words_per_k(int warps, int S) { return xd_window_slots(warps, S) / 8; }
// the origins, padded to whole 32-byte sectors so that every antidiagonal's
// row of words starts on a sector (a kernel may then skip the sectors of a
// row that hold no live slot without partial-sector writes)
FILTR_HD int64_t xd_origin_words(int64_t M, int64_t N) { return (M + N + 1 + 7) & ~(int64_t)7; }
FILTR_HD uint64_t xd_tb_words(int64_t M, int64_t N, int warps, int S) {
  return (uint64_t)xd_origin_words(M, N) + (uint64_t)(M + N + 1) * (uint64_t)xd_words_per_k(warps, S);
}

// Checkpointed sweep of one long pair (filtr_align_long).  The antidiagonals
// are cut into segments (s*C, (s+1)*C].  Mode 3 sweeps one segment forward
// without traceback, resuming from the checkpoint of its first antidiagonal,
// and stores the window state after its last one; the host launches it once
// per group width (1, 2, 4, ... warps) and each launch does nothing if the
// segment is already done, the sweep has finished, or the checkpointed state
// does not fit its window -- so every segment runs at the narrowest width
// that holds it.  Mode 2 resumes from the checkpoint of k_start and recomputes
// (k_start, k_end] with traceback into a segment buffer, which a resumable
// walk then consumes backwards.
struct XdCkpt {
  int mode;            // 3 forward segment, 2 recompute one segment with traceback
  int C;               // checkpoint interval in antidiagonals
  int32_t *buf;        // checkpoints, xd_ckpt_stride() ints each, indexed by k / C
  int k_start, k_end;  // the segment (k_start, k_end]
  uint32_t *seg_tb;    // mode 2: (k_end - k_start) rows of WIN/8 words
  int32_t *seg_ck;     // mode 2: window origin of each recomputed antidiagonal
  int32_t *flags;      // mode 3: [0] sweep finished (2: traceback pool exhausted),
                       //         [1 + s] width that completed segment s
  // mode 3 with traceback (single pass): each attempt at a segment reserves
  // C rows of its window's words from the pool; the attempt that completes
  // the segment records where they are and at which width
  uint32_t *pool;
  uint64_t pool_words;
  unsigned long long *pool_next;
  int32_t *seg_ck_all;  // window origin of every antidiagonal, C per segment
  uint64_t *seg_off;    // per segment: first pool word of its rows
  int32_t *seg_w;       // per segment: its width in warps
};
// checkpoint record: a header, then H, E, F of antidiagonal k and H of k - 1
// for every slot of the widest window (thread t's 4*S values at 16 + t*4*S);
// slots at or beyond the writer's window read as NEG
enum : int {
  XCK_ORIGIN = 0, XCK_DPREV, XCK_BEST, XCK_LO, XCK_HI, XCK_USED, XCK_WIN,
  XCK_BV, XCK_BI, XCK_BJ, XCK_CELLS_LO, XCK_CELLS_HI, XCK_DBEST, XCK_HDR = 16
};
constexpr int XD_MAX_WARPS = 32;
FILTR_HD int64_t xd_ckpt_stride() { return XCK_HDR + (int64_t)xd_window_slots(XD_MAX_WARPS, 8) * 4; }

// Resumable walk over checkpointed segments (one thread).
struct WalkState {
  int i, j, v, state, done, cur;
  uint32_t n, run;
};

#ifdef __CUDACC__
struct XdGeom {
  const int32_t *ck;
  const uint32_t *tb;
  int wpk;
};

__device__ __forceinline__ void xd_geom_init(XdGeom &g, const uint32_t *base, int64_t M, int64_t N,
                                             const TbLayout &L) {
  g.ck = reinterpret_cast<const int32_t *>(base);
  g.tb = base + xd_origin_words(M, N);
  g.wpk = xd_words_per_k(L.warps, L.R);
}

__device__ __forceinline__ uint32_t xd_bits(const XdGeom &g, int i, int j) {
  const int64_t k = (int64_t)i + j;
  const int p = j - __ldg(g.ck + k);
  const uint32_t w = __ldg(g.tb + k * g.wpk + (p >> 3));
  return tb_nibble(w, p);
}
#endif

}  // namespace filtr
