// k_tb.cu -- traceback walk, CIGAR offset scan and CIGAR compaction.
//
// The walk follows the 4-bit choices the forward kernels stored (one nibble per
// cell, see tb_push4 in filtr_internal.h) from
// the end cell back to the start, tracking the current value so that a local
// walk stops on the first H of 0 (Smith-Waterman) and emitting run-length BAM
// ops in reverse into a per-pair staging area.  Global walks that reach row 0
// or column 0 finish with the forced gap.  A scan then places every pair's
// CIGAR in pair order and a warp per pair copies it forward into the caller's
// buffer.
#include "filtr_internal.h"
#include "k_xdrop_layout.h"

namespace filtr {
namespace {

constexpr int OP_I = 1, OP_D = 2, OP_EQ = 7, OP_X = 8;

struct FullGeom {
  int R, HS, M, N;
  bool band;
  int64_t lo, hi;
  int64_t base;   // first word of strip `s`
  int s;          // current strip
  int64_t jlo;    // first column of strip s
  int64_t nsteps; // steps of strip s
};

__device__ __forceinline__ void geom_seek(FullGeom &g, int s) {
  // strips are visited upward only; move `base` from strip g.s to strip s
  while (g.s > s) {
    --g.s;
    int64_t jl, jh;
    strip_cols((int64_t)g.s * g.HS, g.HS, g.M, g.N, g.band, g.lo, g.hi, &jl, &jh);
    g.base -= strip_tb_words(jl, jh, g.R);
    g.jlo = jl;
    g.nsteps = jh >= jl ? (jh - jl + 1) + 31 : 0;
  }
}

// A cursor past the last strip of an M x N int32 tile (strips of 32 * R rows):
// base = the words of every strip, so the first seek moves it down to the strip
// that holds the row asked for.
__device__ __forceinline__ void geom_init(FullGeom &g, int R, int M, int N, const ScoreParams &sp) {
  g.R = R;
  g.HS = 32 * R;
  g.M = M;
  g.N = N;
  g.band = sp.use_band != 0;
  band_limits(M, N, sp.band, sp.band_literal, &g.lo, &g.hi);
  if (!g.band) {
    g.lo = -(int64_t)M - 1;
    g.hi = (int64_t)N + 1;
  }
  const int nstrips = (M + g.HS - 1) / g.HS;
  g.base = 0;
  g.s = nstrips;
  g.jlo = 1;
  g.nsteps = 0;
  for (int s = 0; s < nstrips; ++s) {
    int64_t jl, jh;
    strip_cols((int64_t)s * g.HS, g.HS, M, N, g.band, g.lo, g.hi, &jl, &jh);
    g.base += strip_tb_words(jl, jh, g.R);
  }
}

// Choice bits of cell (i, j) of an int32 tile (banded or not).  The cursor g
// only moves up, so successive calls on one cursor must ask for rows that do
// not increase.
__device__ __forceinline__ uint32_t full_bits(const uint32_t *tb, FullGeom &g, int i, int j) {
  const int s = (i - 1) / g.HS;
  geom_seek(g, s);
  const int rho = (i - 1) - s * g.HS;
  const int l = rho / g.R, k = rho - l * g.R;
  const int64_t t = (int64_t)j - g.jlo + l;
  if (t < 0 || t >= g.nsteps) return 0;  // never taken on a consistent traceback
  const int wps = g.R / 8;
  const uint32_t w = __ldg(tb + g.base + (t * wps + (k >> 3)) * 32 + l);
  return tb_nibble(w, k);
}

// The int16x2 tiled kernel's layout (unbanded): every strip has N + 63 steps
// of 2 * ceil(R/16) words per lane; the high half of a lane's rows runs one step behind.
struct PackGeom {
  int R;
  int64_t strip_words;
};

__device__ __forceinline__ uint32_t pack_bits(const uint32_t *tb, const PackGeom &g, int i, int j) {
  const int HS = 32 * g.R, P = g.R >> 1;
  const int s = (i - 1) / HS;
  const int rho = (i - 1) - s * HS;
  const int l = rho / g.R, kk = rho - l * g.R;
  const int h = kk >= P ? 1 : 0, k = kk - h * P;
  const int64_t t = (int64_t)j - 1 + 2 * l + h;
  const int G = (P + 7) / 8, wps = 2 * G;
  const uint32_t w = __ldg(tb + s * g.strip_words + (t * wps + h * G + (k >> 3)) * 32 + l);
  const int c = k & 7;
  return (((w >> c) & 1u) << 3) | (((w >> (8 + c)) & 1u) << 2) | (((w >> (16 + c)) & 1u) << 1) |
         ((w >> (24 + c)) & 1u);
}

// Choice bits of cell (i, j) of an unbanded int32 tile: every strip has N + 31
// steps of R / 8 words per lane.
__device__ __forceinline__ uint32_t full_bits_unbanded(const uint32_t *tb, int R, int N, int i,
                                                       int j) {
  const int HS = 32 * R, s = (i - 1) / HS, rho = (i - 1) - s * HS;
  const int l = rho / R, k = rho - l * R, wps = R / 8;
  const int64_t t = (int64_t)j - 1 + l;
  const int64_t base = (int64_t)s * strip_tb_words(1, N, R);
  return tb_nibble(__ldg(tb + base + (t * wps + (k >> 3)) * 32 + l), k);
}

struct Emitter {
  uint32_t *st;
  uint32_t n;
  int cur;
  uint32_t run;
  __device__ void put(int op, uint32_t len) {
    if (op == cur) {
      run += len;
    } else {
      if (cur >= 0) st[n++] = (run << 4) | (uint32_t)cur;
      cur = op;
      run = len;
    }
  }
  __device__ void flush() {
    if (cur >= 0) st[n++] = (run << 4) | (uint32_t)cur;
    cur = -1;
  }
};

// One thread walks pair p (any layout).
__device__ __forceinline__ void walk_thread(const WalkArgs &a, const BatchDev &b,
                                            filtr_result *out, uint32_t p) {
  const FwdOut f = a.fwd[p];
  const TbLayout L = a.tbl[p];
  if (f.status != FILTR_ST_OK && f.status != FILTR_ST_DROPPED) {
    out[p].cigar_len = 0;
    return;
  }
  const int M = (int)b.q_len[p], N = (int)b.r_len[p];
  const uint8_t *q = b.q_seq + b.q_off[p];
  const uint8_t *r = b.r_seq + b.r_off[p];
  const bool local = a.sp.mode == FILTR_LOCAL;
  const int A = a.sp.alphabet, e = a.sp.e, oe = a.sp.o + a.sp.e;
  const uint32_t *tb = a.tb + L.off;

  FullGeom g;
  XdGeom xg;
  PackGeom pg{L.R, (int64_t)pack_strip_tb_words(1, N, L.R)};
  if (L.family == FAM_FULL && L.valid) {
    geom_init(g, L.R, M, N, a.sp);
  } else if (L.family == FAM_XDROP && L.valid) {
    xd_geom_init(xg, tb, M, N, L);
  }

  Emitter em{a.stage + a.stage_off[p], 0, -1, 0};
  int i = f.end_i, j = f.end_j, v = f.score, state = 0;
  for (;;) {
    if (state == 0) {
      if (i == 0 && j == 0) break;
      if (local && v == 0) break;
      if (i == 0) {
        em.put(OP_D, (uint32_t)j);
        j = 0;
        break;
      }
      if (j == 0) {
        em.put(OP_I, (uint32_t)i);
        i = 0;
        break;
      }
      const uint32_t nib = (L.family == FAM_FULL)   ? full_bits(tb, g, i, j)
                                 : (L.family == FAM_PACK) ? pack_bits(tb, pg, i, j)
                                                          : xd_bits(xg, i, j);
      if (nib & TB_PF) {
        state = 2;
      } else if (nib & TB_PE) {
        state = 1;
      } else {
        const int qc = q[i - 1], rc = r[j - 1];
        em.put(qc == rc ? OP_EQ : OP_X, 1);
        v -= a.sp.subst[qc * A + rc];
        --i;
        --j;
      }
    } else if (state == 1) {
      if (j == 0) {
        state = 0;
        continue;
      }
      const uint32_t nib = (L.family == FAM_FULL)   ? full_bits(tb, g, i, j)
                                 : (L.family == FAM_PACK) ? pack_bits(tb, pg, i, j)
                                                          : xd_bits(xg, i, j);
      em.put(OP_D, 1);
      if (nib & TB_EEXT) {
        v += e;
      } else {
        v += oe;
        state = a.sp.mid ? 3 : 0;
      }
      --j;
    } else if (state == 2) {
      if (i == 0) {
        state = 0;
        continue;
      }
      const uint32_t nib = (L.family == FAM_FULL)   ? full_bits(tb, g, i, j)
                                 : (L.family == FAM_PACK) ? pack_bits(tb, pg, i, j)
                                                          : xd_bits(xg, i, j);
      em.put(OP_I, 1);
      if (nib & TB_FEXT) {
        v += e;
      } else {
        v += oe;
        state = a.sp.mid ? 3 : 0;
      }
      --i;
    } else {  // state 3 (M/I/D): the gap opened from M here, a diagonal step
      if (i == 0 && j == 0) break;
      const int qc = q[i - 1], rc = r[j - 1];
      em.put(qc == rc ? OP_EQ : OP_X, 1);
      v -= a.sp.subst[qc * A + rc];
      --i;
      --j;
      state = 0;
    }
  }
  em.flush();
  filtr_result *res = out + p;
  res->q_begin = i;
  res->r_begin = j;
  res->cigar_len = em.n;
}

__global__ void k_walk(const WalkArgs a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const GraphDesc *gd = a.gd;  // captured pipeline: batch, outputs and count from here
  if (gd && gd->abort) return;
  if (t >= (gd ? gd->n : a.n_order)) return;
  walk_thread(a, gd ? gd->b : a.b, gd ? gd->out : a.out, a.order[t]);
}

// ---- warp walks over the antidiagonal (X-drop) layout ------------------------
// The walk itself is serial, and one thread per pair spends it waiting on two
// dependent loads per step (the window origin c_k, then the traceback word).
// A warp prefetches instead: from the current cell (i0, j0) on antidiagonal
// k0, lane L loads c of antidiagonal k0 - L and the words holding the slots a
// path from (i0, j0) can reach there -- every step lowers i + j by 1 or 2 and
// j by at most 1, so on k0 - L the path's column lies in [j0 - L, j0]: at most
// 32 slots, 5 words.  Lane 0 then walks through shared memory until the path
// leaves the 32 cached antidiagonals, and the warp refills.

constexpr int XW = 5;  // cached words per antidiagonal

struct WalkCore {
  const uint8_t *q, *r;
  const int8_t *subst;
  int A, e, oe;
  bool local;
  int i, j, v, state;
  Emitter em;
  bool mid = false;  // Table 1's M/I/D: a gap that opened leaves through a diagonal step (state 3)
};

// One step of the walk (those of k_walk): 1 when the alignment's start is
// reached, 2 when the current cell's antidiagonal is <= k_stop or < k_low or
// its bits are not cached (state kept), else 0.  Codes gives the residue codes
// of the diagonal steps (cached by the warp beside the bits).
template <class Bits, class Codes>
__device__ __forceinline__ int walk_step(WalkCore &w, const Bits &bits, int64_t k_stop, int64_t k_low,
                                         const Codes &codes) {
  if (w.state == 0) {
    if ((w.i == 0 && w.j == 0) || (w.local && w.v == 0)) return 1;
    if (w.i == 0) {
      w.em.put(OP_D, (uint32_t)w.j);
      w.j = 0;
      return 1;
    }
    if (w.j == 0) {
      w.em.put(OP_I, (uint32_t)w.i);
      w.i = 0;
      return 1;
    }
  }
  const int64_t k = (int64_t)w.i + w.j;
  if (k <= k_stop || k < k_low) return 2;
  if (w.state == 0) {
    const uint32_t nib = bits(w.i, w.j);
    if (nib > 15u) return 2;  // not cached: the warp refills around (i, j)
    if (nib & TB_PF) {
      w.state = 2;
    } else if (nib & TB_PE) {
      w.state = 1;
    } else {
      const int qc = codes.q(w, w.i), rc = codes.r(w, w.j);
      w.em.put(qc == rc ? OP_EQ : OP_X, 1);
      w.v -= w.subst[qc * w.A + rc];
      --w.i;
      --w.j;
    }
  } else if (w.state == 1) {
    if (w.j == 0) {
      w.state = 0;
      return 0;
    }
    const uint32_t nib = bits(w.i, w.j);
    if (nib > 15u) return 2;
    w.em.put(OP_D, 1);
    if (nib & TB_EEXT) {
      w.v += w.e;
    } else {
      w.v += w.oe;
      w.state = w.mid ? 3 : 0;
    }
    --w.j;
  } else if (w.state == 2) {
    if (w.i == 0) {
      w.state = 0;
      return 0;
    }
    const uint32_t nib = bits(w.i, w.j);
    if (nib > 15u) return 2;
    w.em.put(OP_I, 1);
    if (nib & TB_FEXT) {
      w.v += w.e;
    } else {
      w.v += w.oe;
      w.state = w.mid ? 3 : 0;
    }
    --w.i;
  } else {  // state 3: the gap opened from M here, so this cell is a diagonal step
    if (w.i == 0 && w.j == 0) return 1;
    const int qc = codes.q(w, w.i), rc = codes.r(w, w.j);
    w.em.put(qc == rc ? OP_EQ : OP_X, 1);
    w.v -= w.subst[qc * w.A + rc];
    --w.i;
    --w.j;
    w.state = 0;
  }
  return 0;
}

// Walks until the alignment's start is reached (returns true), or until the
// current cell's antidiagonal is <= k_stop or < k_low or its bits are not
// cached (returns false, state kept), with the whole warp (every lane calls
// it; w is lane 0's).  A
// run of diagonal steps (matches and mismatches, H taken from the diagonal) is
// taken in one go: lane d looks at the cell d steps down the diagonal, a ballot
// finds where the run ends (a gap, row or column 0, the window's edge, or for
// local alignments the first cell of value 0), a warp scan gives the value
// change, and lane 0 emits the run's '=' / 'X' ops.  Lane 0 walks the other
// steps alone.
template <class Bits, class Codes>
__device__ __forceinline__ bool walk_coop(WalkCore &w, const Bits &bits, int64_t k_stop,
                                          int64_t k_low, const Codes &codes) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int i = __shfl_sync(FULL, w.i, 0), j = __shfl_sync(FULL, w.j, 0);
    const int v = __shfl_sync(FULL, w.v, 0), st = __shfl_sync(FULL, w.state, 0);
    if (st == 0) {
      const int ii = i - lane, jj = j - lane;
      const int64_t kk = (int64_t)ii + jj;
      bool ok = ii >= 1 && jj >= 1 && kk > k_stop && kk >= k_low;
      int qc = 0, rc = 1, sc = 0;
      if (ok) {
        ok = (bits(ii, jj) & (TB_PE | TB_PF)) == 0u;
        qc = codes.q(w, ii);
        rc = codes.r(w, jj);
        sc = w.subst[qc * w.A + rc];
      }
      int pre = sc;  // inclusive scan of the scores down the diagonal
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, pre, o);
        if (lane >= o) pre += t;
      }
      if (w.local && v - (pre - sc) == 0) ok = false;  // the value at cell d
      const unsigned okm = __ballot_sync(FULL, ok);
      const int L = (okm == FULL) ? 32 : __ffs(~okm) - 1;
      if (L > 0) {
        const unsigned eqm = __ballot_sync(FULL, qc == rc);
        const int dv = __shfl_sync(FULL, pre, L - 1);
        if (lane == 0) {
          int d = 0;
          while (d < L) {
            const unsigned rest = eqm >> d;
            const bool eq = (rest & 1u) != 0u;
            const unsigned stop = eq ? ~rest : rest;
            const int len = min(stop ? __ffs(stop) - 1 : 32 - d, L - d);
            w.em.put(eq ? OP_EQ : OP_X, (uint32_t)len);
            d += len;
          }
          w.v -= dv;
          w.i -= L;
          w.j -= L;
        }
        continue;
      }
    }
    int r = 0;
    if (lane == 0) r = walk_step(w, bits, k_stop, k_low, codes);
    r = __shfl_sync(FULL, r, 0);
    if (r == 1) return true;
    if (r == 2) return false;
  }
}

struct XdCache {
  uint32_t w[32 * XW];
  int32_t c[32], b[32];
  // the 32 query / reference codes below the window's first cell (i0, j0):
  // qc[x] = q[i0 - 1 - x], rc[x] = r[j0 - 1 - x] (a walk inside the window
  // steps diagonally only from cells with i > i0 - 32, j > j0 - 32)
  uint8_t qc[32], rc[32];
  int32_t i0, j0;
};
struct XdCacheCodes {
  const XdCache *C;
  __device__ int q(const WalkCore &, int i) const { return C->qc[C->i0 - i]; }
  __device__ int r(const WalkCore &, int j) const { return C->rc[C->j0 - j]; }
};

// Where antidiagonal k's window origin and traceback row live.
struct XdRows {  // one pair's own layout or a recomputed segment: row = k - row_off
  const int32_t *ck;
  const uint32_t *tb;
  int wpk;
  int64_t row_off;
  __device__ void at(int64_t k, int &c, const uint32_t *&row, int &w) const {
    const int64_t i = k - row_off;
    c = __ldg(ck + i);
    row = tb + i * wpk;
    w = wpk;
  }
};
struct XdPoolRows {  // single-pass segmented sweep: segment s = (k - 1) / C
  const uint32_t *pool;
  const int32_t *seg_ck_all;
  const uint64_t *seg_off;
  const int32_t *seg_w;
  int C;
  __device__ void at(int64_t k, int &c, const uint32_t *&row, int &w) const {
    const int km = (int)(k - 1);  // antidiagonals stay below 2^31
    const int s = km / C, i = km - s * C;
    w = xd_words_per_k(__ldg(seg_w + s), 8);
    c = __ldg(seg_ck_all + (int64_t)s * C + i);
    row = pool + __ldg(seg_off + s) + (int64_t)i * w;
  }
};

// All lanes: cache antidiagonals k0 - lane (those > k_min) around column j0,
// and the residue codes the walk reads below (i0, j0).
template <class Rows>
__device__ __forceinline__ void xd_fill(XdCache &C, const Rows &rows, int64_t k0, int j0,
                                        int64_t k_min, const WalkCore &w) {
  const int lane = threadIdx.x & 31;
  const int i0 = (int)(k0 - j0);
  C.qc[lane] = (i0 - 1 - lane >= 0) ? w.q[i0 - 1 - lane] : 0;
  C.rc[lane] = (j0 - 1 - lane >= 0) ? w.r[j0 - 1 - lane] : 0;
  if (lane == 0) {
    C.i0 = i0;
    C.j0 = j0;
  }
  const int64_t kk = k0 - lane;
  if (kk > k_min) {
    int c, wpk;
    const uint32_t *row;
    rows.at(kk, c, row, wpk);
    const int plo = max(j0 - lane - c, 0), phi = j0 - c;
    const int w0 = plo >> 3, w1 = min(phi >> 3, wpk - 1);
#pragma unroll
    for (int x = 0; x < XW; ++x)
      if (w0 + x <= w1) C.w[lane * XW + x] = __ldg(row + w0 + x);
    C.c[lane] = c;
    C.b[lane] = w0;
  }
  __syncwarp();
}

struct XdCacheBits {
  const XdCache *C;
  int64_t k0;
  __device__ uint32_t operator()(int ii, int jj) const {
    const int L = (int)(k0 - ((int64_t)ii + jj));
    const int p = jj - C->c[L];
    return tb_nibble(C->w[L * XW + (p >> 3) - C->b[L]], p);
  }
};

// One warp per pair of a batched X-drop call (4 pairs per 128-thread block).
__global__ void __launch_bounds__(128) k_walk_xdw(const WalkArgs a) {
  __shared__ XdCache cache[4];
  __shared__ int8_t s_sub[MAX_ALPHA * MAX_ALPHA];
  for (int x = threadIdx.x; x < a.sp.alphabet * a.sp.alphabet; x += blockDim.x) s_sub[x] = a.sp.subst[x];
  __syncthreads();
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t t = blockIdx.x * 4 + wib;
  if (t >= a.n_order) return;
  const uint32_t p = a.order[t];
  const FwdOut f = a.fwd[p];
  const TbLayout L = a.tbl[p];
  if (f.status != FILTR_ST_OK && f.status != FILTR_ST_DROPPED) {
    if (lane == 0) a.out[p].cigar_len = 0;
    return;
  }
  const int M = (int)a.b.q_len[p], N = (int)a.b.r_len[p];
  const uint32_t *base = a.tb + L.off;
  const int32_t *ck = reinterpret_cast<const int32_t *>(base);
  const uint32_t *tbw = base + xd_origin_words(M, N);
  const int wpk = xd_words_per_k(L.warps, L.R);
  WalkCore w{a.b.q_seq + a.b.q_off[p], a.b.r_seq + a.b.r_off[p], s_sub, a.sp.alphabet,
             a.sp.e, a.sp.o + a.sp.e, a.sp.mode == FILTR_LOCAL, f.end_i, f.end_j, f.score, 0,
             Emitter{a.stage + a.stage_off[p], 0, -1, 0}, a.sp.mid != 0};
  XdCache &C = cache[wib];
  bool done = false;
  for (;;) {
    const int i0 = __shfl_sync(0xffffffffu, w.i, 0), j0 = __shfl_sync(0xffffffffu, w.j, 0);
    if (__shfl_sync(0xffffffffu, (int)done, 0)) break;
    const int64_t k0 = (int64_t)i0 + j0;
    xd_fill(C, XdRows{ck, tbw, wpk, 0}, k0, j0, 0, w);
    done = walk_coop(w, XdCacheBits{&C, k0}, -1, k0 - 31, XdCacheCodes{&C});
    __syncwarp();
  }
  if (lane == 0) {
    w.em.flush();
    filtr_result *res = a.out + p;
    res->q_begin = w.i;
    res->r_begin = w.j;
    res->cigar_len = w.em.n;
  }
}

// ---- warp walk over the tiled layouts ---------------------------------------
// One thread per pair waits on one dependent load per step.  A warp instead
// caches, from the current cell (i0, j0), the choice bits of three lines of 32
// cells: the diagonal (i0 - d, j0 - d), the row (i0, j0 - d) and the column
// (i0 - d, j0) -- lane d loads its three words at once.  Matches and
// mismatches follow the diagonal, a gap the row or the column, so lane 0 walks
// from the cache until the path leaves all three lines (a gap's start or end),
// and the warp refills there: about two refills per gap instead of a load per
// step.  Runs of diagonal steps along the cached diagonal are taken by the
// whole warp (walk_coop), with the 32 codes below (i0, j0) cached beside the
// bits.  In a banded int32 tile the strips' offsets depend on the band, so
// every lane keeps two strip cursors: one for row i0 and one for row i0 - d.
// Both rows never increase from one refill to the next, and a cursor only
// moves up.

struct TileCache {
  uint8_t d[32], row[32], col[32];
  // qc[x] = q[i0 - 1 - x], rc[x] = r[j0 - 1 - x]: the codes of the diagonal
  // line's cells (and of the row's and the column's)
  uint8_t qc[32], rc[32];
  int32_t i0, j0;
};
struct TileCacheCodes {  // cached codes; cells further from (i0, j0) read the sequences
  const TileCache *C;
  __device__ int q(const WalkCore &w, int i) const {
    const int x = C->i0 - i;
    return x < 32 ? C->qc[x] : w.q[i - 1];
  }
  __device__ int r(const WalkCore &w, int j) const {
    const int x = C->j0 - j;
    return x < 32 ? C->rc[x] : w.r[j - 1];
  }
};

struct TileCacheBits {
  const TileCache *C;
  int i0, j0;
  __device__ uint32_t operator()(int ii, int jj) const {
    const int di = i0 - ii, dj = j0 - jj;
    if (di == dj && di < 32) return C->d[di];
    if (di == 0 && dj < 32) return C->row[dj];
    if (dj == 0 && di < 32) return C->col[di];
    return 0xffu;  // not cached
  }
};

__global__ void __launch_bounds__(128) k_walk_tw(const WalkArgs a) {
  __shared__ TileCache cache[4];
  __shared__ int8_t s_sub[MAX_ALPHA * MAX_ALPHA];
  for (int x = threadIdx.x; x < a.sp.alphabet * a.sp.alphabet; x += blockDim.x) s_sub[x] = a.sp.subst[x];
  __syncthreads();
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t t = blockIdx.x * 4 + wib;
  const GraphDesc *gd = a.gd;  // captured pipeline: batch, outputs and count from here
  if (gd && gd->abort) return;
  if (t >= (gd ? gd->n : a.n_order)) return;
  const BatchDev b = gd ? gd->b : a.b;
  filtr_result *const out = gd ? gd->out : a.out;
  const uint32_t p = a.order[t];
  const TbLayout L = a.tbl[p];
  const bool pk = L.family == FAM_PACK;
  if (!L.valid || !(pk || L.family == FAM_FULL)) {
    if (lane == 0) walk_thread(a, b, out, p);  // empty pairs
    return;
  }
  const bool fb = !pk && a.sp.use_band;
  const FwdOut f = a.fwd[p];
  if (f.status != FILTR_ST_OK && f.status != FILTR_ST_DROPPED) {
    if (lane == 0) out[p].cigar_len = 0;
    return;
  }
  const int N = (int)b.r_len[p];
  const uint32_t *tb = a.tb + L.off;
  const PackGeom pg{L.R, (int64_t)pack_strip_tb_words(1, N, L.R)};
  WalkCore w{b.q_seq + b.q_off[p], b.r_seq + b.r_off[p], s_sub, a.sp.alphabet,
             a.sp.e, a.sp.o + a.sp.e, a.sp.mode == FILTR_LOCAL, f.end_i, f.end_j, f.score, 0,
             Emitter{a.stage + a.stage_off[p], 0, -1, 0}, a.sp.mid != 0};
  TileCache &C = cache[wib];
  bool done = false;
  FullGeom g_row, g_lane;  // banded int32 tiles: cursors for rows i0 and i0 - lane
  if (fb) {
    geom_init(g_row, L.R, (int)b.q_len[p], N, a.sp);
    g_lane = g_row;
  }
  auto cell = [&](FullGeom &g, int ii, int jj) -> uint8_t {
    if (ii < 1 || jj < 1) return 0;
    if (pk) return (uint8_t)pack_bits(tb, pg, ii, jj);
    if (fb) return (uint8_t)full_bits(tb, g, ii, jj);
    return (uint8_t)full_bits_unbanded(tb, L.R, N, ii, jj);
  };
  for (;;) {
    const int i0 = __shfl_sync(0xffffffffu, w.i, 0), j0 = __shfl_sync(0xffffffffu, w.j, 0);
    if (__shfl_sync(0xffffffffu, (int)done, 0)) break;
    const uint8_t cr = cell(g_row, i0, j0 - lane), cd = cell(g_lane, i0 - lane, j0 - lane),
                  cc = cell(g_lane, i0 - lane, j0);
    C.d[lane] = cd;
    C.row[lane] = cr;
    C.col[lane] = cc;
    C.qc[lane] = (i0 - 1 - lane >= 0) ? w.q[i0 - 1 - lane] : 0;
    C.rc[lane] = (j0 - 1 - lane >= 0) ? w.r[j0 - 1 - lane] : 0;
    if (lane == 0) {
      C.i0 = i0;
      C.j0 = j0;
    }
    __syncwarp();
    done = walk_coop(w, TileCacheBits{&C, i0, j0}, -1, INT64_MIN, TileCacheCodes{&C});
    __syncwarp();
  }
  if (lane == 0) {
    w.em.flush();
    filtr_result *res = out + p;
    res->q_begin = w.i;
    res->r_begin = w.j;
    res->cigar_len = w.em.n;
  }
}

// Resumable walk over one recomputed segment (antidiagonals (k_start, k_end])
// of a checkpointed X-drop traceback; one warp.  Stops when the walk leaves
// the segment (the next, earlier segment continues from the saved state) or
// when the alignment's start is reached.
__global__ void k_walk_segw(const WalkArgs a, const uint32_t *seg_tb, const int32_t *seg_ck,
                            int k_start, int wpk, WalkState *ws) {
  __shared__ XdCache C;
  __shared__ int8_t s_sub[MAX_ALPHA * MAX_ALPHA];
  for (int x = threadIdx.x; x < a.sp.alphabet * a.sp.alphabet; x += blockDim.x) s_sub[x] = a.sp.subst[x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const WalkState st = *ws;
  if (st.done) return;
  const uint32_t p = a.order[0];
  WalkCore w{a.b.q_seq + a.b.q_off[p], a.b.r_seq + a.b.r_off[p], s_sub, a.sp.alphabet,
             a.sp.e, a.sp.o + a.sp.e, a.sp.mode == FILTR_LOCAL, st.i, st.j, st.v, st.state,
             Emitter{a.stage + a.stage_off[p], st.n, st.cur, st.run}, a.sp.mid != 0};
  bool done = false;
  for (;;) {
    const int i0 = __shfl_sync(0xffffffffu, w.i, 0), j0 = __shfl_sync(0xffffffffu, w.j, 0);
    const bool d = __shfl_sync(0xffffffffu, (int)done, 0) != 0;
    const int64_t k0 = (int64_t)i0 + j0;
    if (d || k0 <= k_start) break;
    xd_fill(C, XdRows{seg_ck, seg_tb, wpk, (int64_t)k_start + 1}, k0, j0, k_start, w);
    done = walk_coop(w, XdCacheBits{&C, k0}, k_start, k0 - 31, XdCacheCodes{&C});
    __syncwarp();
  }
  if (lane == 0) {
    if (done) {
      w.em.flush();
      filtr_result *res = a.out + p;
      res->q_begin = w.i;
      res->r_begin = w.j;
      res->cigar_len = w.em.n;
    }
    WalkState o;
    o.i = w.i;
    o.j = w.j;
    o.v = w.v;
    o.state = w.state;
    o.done = done ? 1 : 0;
    o.n = w.em.n;
    o.cur = w.em.cur;
    o.run = w.em.run;
    *ws = o;
  }
}

// The whole traceback of a single-pass segmented sweep; one warp.
__global__ void k_walk_poolw(const WalkArgs a, const XdPoolRows rows) {
  __shared__ XdCache C;
  __shared__ int8_t s_sub[MAX_ALPHA * MAX_ALPHA];
  for (int x = threadIdx.x; x < a.sp.alphabet * a.sp.alphabet; x += blockDim.x) s_sub[x] = a.sp.subst[x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const uint32_t p = a.order[0];
  const FwdOut f = a.fwd[p];
  if (f.status != FILTR_ST_OK && f.status != FILTR_ST_DROPPED) {
    if (lane == 0) a.out[p].cigar_len = 0;
    return;
  }
  WalkCore w{a.b.q_seq + a.b.q_off[p], a.b.r_seq + a.b.r_off[p], s_sub, a.sp.alphabet,
             a.sp.e, a.sp.o + a.sp.e, a.sp.mode == FILTR_LOCAL, f.end_i, f.end_j, f.score, 0,
             Emitter{a.stage + a.stage_off[p], 0, -1, 0}, a.sp.mid != 0};
  bool done = false;
  for (;;) {
    const int i0 = __shfl_sync(0xffffffffu, w.i, 0), j0 = __shfl_sync(0xffffffffu, w.j, 0);
    if (__shfl_sync(0xffffffffu, (int)done, 0)) break;
    const int64_t k0 = (int64_t)i0 + j0;
    xd_fill(C, rows, k0, j0, 0, w);
    done = walk_coop(w, XdCacheBits{&C, k0}, -1, k0 - 31, XdCacheCodes{&C});
    __syncwarp();
  }
  if (lane == 0) {
    w.em.flush();
    filtr_result *res = a.out + p;
    res->q_begin = w.i;
    res->r_begin = w.j;
    res->cigar_len = w.em.n;
  }
}

// Exclusive scan of cigar_len (pair order) into offs; *total = sum.  One CTA.
__global__ void k_scan(const filtr_result *out, uint32_t n, uint64_t *offs, uint64_t *total,
                       const GraphDesc *gd) {
  __shared__ uint64_t part[1024];
  __shared__ uint64_t carry;
  if (gd) {  // captured pipeline (uniform over the block)
    if (gd->abort) return;
    out = gd->out;
    n = gd->n;
  }
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  constexpr int PER = 8;
  for (uint64_t base = 0; base < n; base += (uint64_t)blockDim.x * PER) {
    uint64_t v[PER];
    uint64_t sum = 0;
    const uint64_t b0 = base + (uint64_t)threadIdx.x * PER;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      v[k] = (b0 + k < n) ? out[b0 + k].cigar_len : 0;
      sum += v[k];
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      uint64_t add = (threadIdx.x >= (unsigned)off) ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    uint64_t run = carry + part[threadIdx.x] - sum;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      if (b0 + k < n) offs[b0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// One warp per pair: reverse the staged ops into the caller's buffer.
__global__ void k_compact(const WalkArgs a, uint32_t n, const uint64_t *offs, uint32_t *cigar,
                          uint64_t cap, filtr_result *out) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a.gd) {  // captured pipeline
    if (a.gd->abort) return;
    n = a.gd->n;
    cigar = a.gd->cigar;
    cap = a.gd->cap;
    out = a.gd->out;
  }
  if (w >= n) return;
  const uint32_t len = out[w].cigar_len;
  const uint64_t off = offs[w];
  if (lane == 0) out[w].cigar_off = off;
  if (len == 0 || cigar == nullptr || off + len > cap) return;
  const uint32_t *st = a.stage + a.stage_off[w];
  for (uint32_t x = lane; x < len; x += 32) cigar[off + x] = st[len - 1 - x];
}

}  // namespace

cudaError_t launch_walk(const WalkArgs &a, cudaStream_t s) {
  if (a.n_order == 0) return cudaSuccess;
  // A warp per pair keeps more loads in flight for each pair but issues the
  // serial walk as a whole warp's instructions: for one or a few pairs (plain
  // per-pair calls, a long pair) it is the faster form; with thousands of pairs
  // a thread per pair (32 pairs per instruction stream) is (2.5 ms against
  // 3.4 ms for the 100,000-pair protein batch).
  if (a.n_order <= 256)
    k_walk_tw<<<(a.n_order + 3) / 4, 128, 0, s>>>(a);
  else
    k_walk<<<(a.n_order + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}


cudaError_t launch_walk_xd(const WalkArgs &a, cudaStream_t s) {
  if (a.n_order == 0) return cudaSuccess;
  k_walk_xdw<<<(a.n_order + 3) / 4, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_walk_pool(const WalkArgs &a, const uint32_t *pool, const int32_t *seg_ck_all,
                             const uint64_t *seg_off, const int32_t *seg_w, int C, cudaStream_t s) {
  k_walk_poolw<<<1, 32, 0, s>>>(a, XdPoolRows{pool, seg_ck_all, seg_off, seg_w, C});
  return cudaGetLastError();
}

cudaError_t launch_walk_segment(const WalkArgs &a, const uint32_t *seg_tb, const int32_t *seg_ck,
                                int k_start, int wpk, WalkState *st, cudaStream_t s) {
  k_walk_segw<<<1, 32, 0, s>>>(a, seg_tb, seg_ck, k_start, wpk, st);
  return cudaGetLastError();
}

cudaError_t launch_scan_offsets(const filtr_result *out, uint32_t n, uint64_t *offs,
                                uint64_t *total, cudaStream_t s, const GraphDesc *gd) {
  k_scan<<<1, 1024, 0, s>>>(out, n, offs, total, gd);
  return cudaGetLastError();
}

cudaError_t launch_compact(const WalkArgs &a, uint32_t n, const uint64_t *offs, uint32_t *cigar,
                           uint64_t cap, filtr_result *out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t threads = (uint64_t)n * 32;
  k_compact<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, n, offs, cigar, cap, out);
  return cudaGetLastError();
}

}  // namespace filtr
