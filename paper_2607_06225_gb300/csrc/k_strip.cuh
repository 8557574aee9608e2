// k_strip.cuh -- one row strip of the tiled wavefront (shared by the batched
// kernel k_full and the intra-pair kernel k_long).
//
// A strip is 32*R query rows; lane l owns rows [row0 + lR + 1, row0 + lR + R]
// in registers.  At step t lane l updates column j = jlo + t - l of its rows,
// so the warp's active cells form a staircase along the antidiagonal
// direction: every dependency of a lane's top row (left: own registers, up:
// lane l-1's bottom row at the same column, diagonal: lane l-1's bottom row one
// column back) was produced at the previous step and arrives by one
// __shfl_up_sync.  Rows inside a lane are updated top to bottom.  This is the
// antidiagonal order of Sec. 6.2 applied to R-row tiles; reordering never
// changes values or traceback (Sec. 6).  Lane 0 reads the strip above's bottom
// row (H, F per column) through the IO object; lane 31 writes this strip's.
//
// Cell update (affine, Gotoh H/E/F), plain int32 add / max:
//   E = max(E_left - e, H_left - (o+e))
//   F = max(F_up - e, H_up - (o+e))
//   H = max(max(H_diag + s, E), F) [, 0]
// Plain adds issue on the FMA pipe (written as multiply-adds) and maxima on
// the ALU pipe; a DPX add-max (__viaddmax_s32) or three-way max (__vimax3_s32)
// takes one ALU slot for two operations (filtr_probe_int_peak measures both
// rates).  E and F use the add-max and the traceback's extension bits come from
// H - (o+e) - E and H - (o+e) - F, which balances the two pipes at about 8.5
// instructions each per affine traceback cell.  Substitution scores come from
// a per-strip query profile in shared memory (profile[a][row] = s(q_row, a)):
// one 8- or 16-byte load per lane per step.
//
// Traceback: 4 bits per cell, each the sign of a difference shifted into the
// lane's word (tb_push4): E > D, F > max(D, E), E took the extension, F took the
// extension.  Cell k of a word ends in bits [4*(7 - k), 4*(7 - k) + 4).  Per
// strip: step-major, then word (R/8 per lane), then lane.
#pragma once

#include <climits>

#include "filtr_internal.h"

namespace filtr {

constexpr unsigned STRIP_FULLMASK = 0xffffffffu;

template <int R>
struct ProfWord;
template <>
struct ProfWord<8> {
  using T = uint2;
};
template <>
struct ProfWord<16> {
  using T = uint4;
};
struct alignas(8) Prof24 {
  uint2 a, b, c;
};
template <>
struct ProfWord<24> {
  using T = Prof24;
};
struct alignas(16) Prof32 {
  uint4 a, b;
};
template <>
struct ProfWord<32> {
  using T = Prof32;
};

// Signed byte B of a word, sign-extended by one PTX byte permute: selector
// nibble B copies byte B, nibbles with the msb set replicate its sign bit.
// (__byte_perm ignores the selector msb, so it cannot do this.)
template <int B>
__device__ __forceinline__ int sext_byte(uint32_t w) {
  constexpr uint32_t sel = B | ((8u | B) << 4) | ((8u | B) << 8) | ((8u | B) << 12);
  int r;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(w), "n"(sel));
  return r;
}

template <int R>
__device__ __forceinline__ void unpack_scores(const typename ProfWord<R>::T &w, int (&sc)[R]) {
  const uint32_t *u = reinterpret_cast<const uint32_t *>(&w);
#pragma unroll
  for (int k = 0; k < R / 4; ++k) {
    sc[4 * k + 0] = sext_byte<0>(u[k]);
    sc[4 * k + 1] = sext_byte<1>(u[k]);
    sc[4 * k + 2] = sext_byte<2>(u[k]);
    sc[4 * k + 3] = sext_byte<3>(u[k]);
  }
}

// a + b * one with `one` == 1 held in a register the compiler cannot fold:
// the add issues as an integer multiply-add on the FMA pipe, leaving the ALU
// pipe to the max, funnel-shift and byte-permute work of the cell update (the
// two pipes issue in parallel; the kernel is otherwise ALU-pipe bound).
__device__ __forceinline__ int fadd(int a, int b, int one) {
  int r;
  asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(one), "r"(a));
  return r;
}
// a - b the same way (mone == -1)
__device__ __forceinline__ int fsub(int a, int b, int mone) { return fadd(a, b, mone); }
// a * b + c on the FMA pipe
__device__ __forceinline__ int fmad(int a, int b, int c) {
  int r;
  asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// Per-pair constants of a strip pass.
struct StripPair {
  int one;           // 1, computed at run time (see fadd)
  int M, N;
  const uint8_t *q, *r;
  int lo, hi;        // band on d = j - i (unbanded: -M-1, N+1)
  int o, e;          // o = 0 for linear gaps
  int A;
  const int8_t *s_sub;  // shared-memory substitution table
  int8_t *prof;         // this warp's profile area (A * 32R bytes)
  uint32_t *tb;         // this pair's traceback words (nullptr without traceback)
};

// Running best cell of a lane (local mode): largest H, then smallest i, then j.
struct LaneBest {
  int v, i, j;
};

// Process strip s.  IO must provide (called by every lane unless noted):
//   bool wait(int j)          -- before lane 0 reads column j of the strip
//                                above; false aborts the strip (timeout)
//   int2 in(int j)            -- lane 0 only: (H, F) of the strip above
//   FETCH                     -- constexpr bool: lane 0's input row is
//                                fetched ahead with fetch() instead of in()
//   int fetch(int j, int jmax, int2 &v) -- (FETCH only) after wait(j): lane x
//                                loads (H, F) of column j + x of the strip
//                                above for the n columns (1 <= n <= 32, up to
//                                jmax) known to be ready; returns n
//   void out(int j, int H, int F) -- lane 31 only: this strip's bottom row
//   void done_col(int j, int jlo, int jhi) -- lane 31 only, after out(j)
// prev_jlo / prev_jhi: the strip above's columns (empty for s == 0).
// Returns false if IO aborted.  endH receives H(M, jhi) for the lane holding
// row M when this is the last strip.
template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND, class IO>
__device__ __forceinline__ bool strip_pass(const StripPair &P, int s, int jlo, int jhi, int prev_jlo,
                                           int prev_jhi, int64_t tb_base, IO &io, LaneBest &best,
                                           int &endH) {
  constexpr int HS = 32 * R;
  constexpr int WPS = R / 8;
  using PW = typename ProfWord<R>::T;
  const int lane = threadIdx.x & 31;
  const int M = P.M, lo = P.lo, hi = P.hi, o = P.o, e = P.e;
  const int one = P.one, mone = -P.one, me = -P.e, moe = -(P.o + P.e);
  const int row0 = s * HS;
  const int top = row0 + lane * R + 1;
  const int nstrips = (M + HS - 1) / HS;

  // query profile of this strip: prof[a * HS + row] = s(q[row0 + row], a);
  // rows past M score -128 against everything (see the best-cell tracking)
  {
    int qc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int row = top - 1 + k;
      qc[k] = (row < M) ? (int)P.q[row] : -1;
    }
    __syncwarp();
    for (int aa = 0; aa < P.A; ++aa) {
      uint32_t *dst = reinterpret_cast<uint32_t *>(P.prof + aa * HS + lane * R);
#pragma unroll
      for (int w = 0; w < R / 4; ++w) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int c = qc[4 * w + b];
          const uint32_t sv = (c >= 0) ? (uint32_t)(uint8_t)P.s_sub[c * P.A + aa] : 0x80u;
          v |= sv << (8 * b);
        }
        dst[w] = v;
      }
    }
    __syncwarp();
  }

  // state of column jlo - 1
  int Hc[R], Ec[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = top + k;
    int h = NEG;
    if (jlo == 1 && (!BAND || -i >= lo)) h = LOCAL ? 0 : -(o + i * e);
    Hc[k] = h;
    Ec[k] = NEG;
  }
  int dtop = NEG;  // H(top - 1, jlo - 1)
  if (jlo == 1) {
    const int i = top - 1;
    if (!BAND || -i >= lo) dtop = (i == 0 || LOCAL) ? 0 : -(o + i * e);
  } else if (s > 0) {
    const int jj = jlo - 1;
    if (jj >= prev_jlo && jj <= prev_jhi) {
      if (!io.wait(jj)) return false;
      if (lane == 0) dtop = io.in(jj).x;
    }
  }

  const int nsteps = (jhi - jlo + 1) + 31;
  int upH = NEG, upF = NEG, prevIn = dtop;
  // lane 0's input row, fetched ahead (IO::FETCH): lane x of pv holds column
  // pbase + x of the strip above (x < pn), so a step waits on a load once per
  // fetch.  A strip that follows the strip above closely (one long pair) would
  // otherwise wait on a load every step; with many warps per SM (batched
  // pairs) the loads' latency is hidden anyway, and the registers cost more.
  int2 pv = make_int2(NEG, NEG);
  int pbase = 0, pn = 0;
  int rc_next = P.r[jlo - 1];
  // Best cell (local), without a per-step scan: each cell's key is
  // H * 32 + (31 - its row in the lane), so the largest key is the largest H
  // and, among equal H, the smallest i; a lane keeps its best key and takes a
  // step's largest key only if strictly greater, so among equal keys (same
  // cell row, later column) the smallest j stays.  A cell of an earlier strip
  // beats an equal H here: the key starts at best.v * 32 + 31.  Keys need
  // H < 2^26 (the host rejects local pairs whose bound reaches it).
  int bestkey = best.v * 32 + 31;
  const int k32 = 32 * P.one;
  for (int t = 0; t < nsteps; ++t) {
    const int j = jlo + t - lane;
    const int j0 = jlo + t;  // lane 0's column
    const bool need = s > 0 && j0 <= jhi && j0 >= prev_jlo && j0 <= prev_jhi;  // warp-uniform
    int2 vin = make_int2(NEG, NEG);
    if constexpr (IO::FETCH) {
      if (need) {
        if (j0 >= pbase + pn) {
          if (!io.wait(j0)) return false;
          pn = io.fetch(j0, prev_jhi, pv);
          pbase = j0;
        }
        vin.x = __shfl_sync(STRIP_FULLMASK, pv.x, j0 - pbase);
        vin.y = AFFINE ? __shfl_sync(STRIP_FULLMASK, pv.y, j0 - pbase) : NEG;
      }
    } else {
      if (need && !io.wait(j0)) return false;
    }
    int inH = __shfl_up_sync(STRIP_FULLMASK, upH, 1);
    int inF = AFFINE ? __shfl_up_sync(STRIP_FULLMASK, upF, 1) : NEG;
    if (lane == 0) {
      if (s == 0) {
        inH = (!BAND || j <= hi) ? (LOCAL ? 0 : -(o + j * e)) : NEG;
        inF = NEG;
      } else if (need) {
        if constexpr (!IO::FETCH) vin = io.in(j);
        inH = vin.x;
        inF = vin.y;
      } else {
        inH = NEG;
        inF = NEG;
      }
    }
    if (j >= jlo && j <= jhi) {
      const int rc = rc_next;
      if (j < jhi) rc_next = P.r[j];
      const PW pw = *reinterpret_cast<const PW *>(P.prof + rc * HS + lane * R);
      int sc[R];
      unpack_scores<R>(pw, sc);
      int Hup = inH, Fup = inF, Hdg = prevIn;
      uint32_t tbw[WPS > 0 ? WPS : 1];
#pragma unroll
      for (int w = 0; w < WPS; ++w) tbw[w] = 0;
      int mkey = 0, kprev = 0;  // largest key of this lane's cells in this column (local mode)
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int Hl = Hc[k];
        const int D = fadd(Hdg, sc[k], one);
        int E, F, H;
        if (AFFINE) {
          const int Hol = fadd(Hl, moe, one), Hou = fadd(Hup, moe, one);
          E = __viaddmax_s32(Ec[k], me, Hol);  // DPX add-max: one ALU slot
          F = __viaddmax_s32(Fup, me, Hou);
          const int DE = max(D, E);
          H = LOCAL ? __vimax3_s32(DE, F, 0) : max(DE, F);  // DPX: one ALU slot
          // E took the extension iff E_left - e > H_left - (o+e) iff E != Hol
          // (a tie keeps the open), so Hol - E < 0 carries the bit
          if (TB)
            tb_push4(tbw[k >> 3], fsub(D, E, mone), fsub(DE, F, mone), fsub(Hol, E, mone),
                     fsub(Hou, F, mone));
        } else {
          E = fadd(Hl, me, one);
          F = fadd(Hup, me, one);
          const int DE = max(D, E);
          H = LOCAL ? __vimax3_s32(DE, F, 0) : max(DE, F);
          if (TB) tb_push4(tbw[k >> 3], fsub(D, E, mone), fsub(DE, F, mone), 0, 0);
        }
        if (BAND) {
          const int dd = j - (top + k);
          if (dd < lo || dd > hi) {
            H = NEG;
            E = NEG;
            F = NEG;
          }
        }
        if (LOCAL) {  // keys of two rows fold into the column's max at once
          const int key = fmad(BAND ? max(H, 0) : H, k32, 31 - k);
          if (k & 1)
            mkey = __vimax3_s32(mkey, kprev, key);
          else
            kprev = key;
        }
        Hdg = Hl;
        Hc[k] = H;
        Ec[k] = E;
        Hup = H;
        Fup = F;
      }
      upH = Hup;
      upF = Fup;
      prevIn = inH;
      if (TB) {
#pragma unroll
        for (int w = 0; w < WPS; ++w) P.tb[tb_base + ((int64_t)t * WPS + w) * 32 + lane] = tbw[w];
      }
      if (lane == 31 && s + 1 < nstrips) {
        io.out(j, Hup, Fup);
        io.done_col(j, jlo, jhi);
      }
      // rows past M stay below a valid cell of their lane already seen, so
      // they never win; lanes wholly past M keep no best
      if (LOCAL && top <= M && mkey > bestkey) {
        bestkey = mkey;
        best.v = mkey >> 5;
        best.i = top + 31 - (mkey & 31);
        best.j = j;
      }
    }
  }
  if (!LOCAL && s == nstrips - 1 && top <= M && M < top + R) {
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (top + k == M) endH = Hc[k];
  }
  __syncwarp();
  return true;
}

// warp-wide reduction of LaneBest with the tie-break (all lanes get the result)
__device__ __forceinline__ LaneBest warp_best(LaneBest b) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const int ov = __shfl_xor_sync(STRIP_FULLMASK, b.v, off);
    const int oi = __shfl_xor_sync(STRIP_FULLMASK, b.i, off);
    const int oj = __shfl_xor_sync(STRIP_FULLMASK, b.j, off);
    if (ov > b.v || (ov == b.v && (oi < b.i || (oi == b.i && oj < b.j)))) {
      b.v = ov;
      b.i = oi;
      b.j = oj;
    }
  }
  return b;
}

}  // namespace filtr
