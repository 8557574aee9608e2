// k_full.cu -- tiled wavefront kernel for full-matrix and statically banded
// alignment (Sec. 2 recurrence; Sec. 7.1 band), with 4-bit traceback.
//
// Schedule.  One warp aligns one pair at a time, pulling pairs from a work
// queue (persistent grid).  The query is cut into strips of 32*R rows; lane l
// owns rows [32R*s + lR + 1, 32R*s + lR + R] of strip s in registers.  At step t
// lane l updates column j = jlo + t - l of its rows, so the warp's active cells
// form a staircase along the antidiagonal direction: every dependency of a
// lane's top row (left: own registers, up: lane l-1's bottom row at the same
// column, diagonal: lane l-1's bottom row one column back) was produced at the
// previous step and arrives by one __shfl_up_sync.  Rows inside a lane are
// updated top to bottom.  This is the antidiagonal order of Sec. 6.2 applied
// to R-row tiles; reordering never changes values or traceback (Sec. 6).
// The strip's bottom row (H and F per column) goes to a per-warp global
// buffer that the next strip's lane 0 reads back.
//
// Cell update (affine, Gotoh H/E/F), plain int32 add / max:
//   E = max(E_left - e, H_left - (o+e))
//   F = max(F_up - e, H_up - (o+e))
//   H = max(max(H_diag + s, E), F) [, 0]
// The DPX forms (__viaddmax_s32, __vimax3_s32) compute the same values but
// issue at half the plain integer rate on sm_103 (filtr_probe_int_peak
// measures both), so the plain forms are used.
// Substitution scores come from a per-strip query profile in shared memory
// (profile[a][row] = s(q_row, a)): one 8- or 16-byte load per lane per step.
//
// Traceback: 4 bits per cell, each the sign of a difference shifted into the
// lane's word (tb_push4, see filtr_internal.h): E > D, F > max(D, E), E took the
// extension, F took the extension.  Cell k of a word ends in bits
// [4*(7 - k), 4*(7 - k) + 4).  Layout per pair: strips in order; per strip,
// step-major, then word (R/8 per lane), then lane.
#include <climits>

#include "filtr_internal.h"

namespace filtr {
namespace {

constexpr unsigned FULLMASK = 0xffffffffu;

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

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND>
__global__ void __launch_bounds__(FULL_WARPS * 32) k_full(const FullArgs a) {
  constexpr int HS = 32 * R;
  constexpr int WPS = R / 8;
  using PW = typename ProfWord<R>::T;
  extern __shared__ __align__(16) int8_t smem[];
  const int A = a.sp.alphabet;
  int8_t *s_sub = smem;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int8_t *prof = smem + 512 + wib * (A * HS);
  for (int t = threadIdx.x; t < A * A; t += blockDim.x) s_sub[t] = a.sp.subst[t];
  __syncthreads();
  const int gw = blockIdx.x * FULL_WARPS + wib;
  int2 *sbuf = a.strip_buf + (size_t)gw * a.strip_stride;
  const int o = a.sp.o, e = a.sp.e, oe = o + e;

  for (;;) {
    uint32_t t0 = 0;
    if (lane == 0) t0 = atomicAdd(a.counter, 1u);
    t0 = __shfl_sync(FULLMASK, t0, 0);
    if (t0 >= a.n_order) break;
    const uint32_t p = a.order[t0];
    const int M = (int)a.b.q_len[p], N = (int)a.b.r_len[p];
    const uint8_t *q = a.b.q_seq + a.b.q_off[p];
    const uint8_t *r = a.b.r_seq + a.b.r_off[p];
    int lo = -M - 1, hi = N + 1;
    if (BAND) {
      int64_t l64, h64;
      band_limits(M, N, a.sp.band, a.sp.band_literal, &l64, &h64);
      lo = (int)(l64 < -(int64_t)M - 1 ? -(int64_t)M - 1 : l64);
      hi = (int)(h64 > (int64_t)N + 1 ? (int64_t)N + 1 : h64);
    }
    const int nstrips = (M + HS - 1) / HS;
    int bestv = 0, besti = INT_MAX, bestj = INT_MAX;
    int endH = NEG;
    uint32_t *tbp = nullptr;
    if (TB) tbp = a.tb + a.tbl[p].off;
    int64_t tb_base = 0;
    int prev_jlo = 1, prev_jhi = 0;

    for (int s = 0; s < nstrips; ++s) {
      const int row0 = s * HS;
      int64_t jl64, jh64;
      strip_cols(row0, HS, M, N, BAND, lo, hi, &jl64, &jh64);
      const int jlo = (int)jl64, jhi = (int)jh64;
      if (jlo > jhi) break;  // no band cell in this strip or below
      const int top = row0 + lane * R + 1;

      // query profile of this strip: prof[a * HS + row] = s(q[row0 + row], a)
      {
        // rows past M score -128 against everything: their values stay below
        // the running best of valid rows (see the best-cell tracking below)
        int qc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int row = top - 1 + k;
          qc[k] = (row < M) ? (int)q[row] : -1;
        }
        __syncwarp();
        for (int aa = 0; aa < A; ++aa) {
          uint32_t *dst = reinterpret_cast<uint32_t *>(prof + aa * HS + lane * R);
#pragma unroll
          for (int w = 0; w < R / 4; ++w) {
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int c = qc[4 * w + b];
              const uint32_t sv = (c >= 0) ? (uint32_t)(uint8_t)s_sub[c * A + aa] : 0x80u;
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
      } else if (lane == 0 && s > 0) {
        const int jj = jlo - 1;
        dtop = (jj >= prev_jlo && jj <= prev_jhi) ? sbuf[jj].x : NEG;
      }

      const int nsteps = (jhi - jlo + 1) + 31;
      int upH = NEG, upF = NEG, prevIn = dtop;
      // prefetch of the residue (and the strip-above row for lane 0) one step ahead
      int rc_next = r[jlo - 1];
      for (int t = 0; t < nsteps; ++t) {
        const int j = jlo + t - lane;
        int inH = __shfl_up_sync(FULLMASK, upH, 1);
        int inF = AFFINE ? __shfl_up_sync(FULLMASK, upF, 1) : NEG;
        if (lane == 0) {
          if (s == 0) {
            inH = (!BAND || j <= hi) ? (LOCAL ? 0 : -(o + j * e)) : NEG;
            inF = NEG;
          } else if (j >= prev_jlo && j <= prev_jhi) {
            const int2 v = sbuf[j];
            inH = v.x;
            inF = v.y;
          } else {
            inH = NEG;
            inF = NEG;
          }
        }
        if (j >= jlo && j <= jhi) {
          const int rc = rc_next;
          if (j < jhi) rc_next = r[j];
          const PW pw = *reinterpret_cast<const PW *>(prof + rc * HS + lane * R);
          int sc[R];
          unpack_scores<R>(pw, sc);
          int Hup = inH, Fup = inF, Hdg = prevIn;
          uint32_t tbw[WPS > 0 ? WPS : 1];
#pragma unroll
          for (int w = 0; w < WPS; ++w) tbw[w] = 0;
          int m = 0;  // column max of this lane's cells (local mode)
#pragma unroll
          for (int k = 0; k < R; ++k) {
            const int Hl = Hc[k];
            const int D = Hdg + sc[k];
            int E, F, H;
            if (AFFINE) {
              const int Hol = Hl - oe, Eext = Ec[k] - e;
              const int Hou = Hup - oe, Fext = Fup - e;
              E = max(Hol, Eext);
              F = max(Hou, Fext);
              const int DE = max(D, E);
              H = max(DE, F);
              if (LOCAL) H = max(H, 0);
              if (TB) tb_push4(tbw[k >> 3], D - E, DE - F, Hol - Eext, Hou - Fext);
            } else {
              E = Hl - e;
              F = Hup - e;
              const int DE = max(D, E);
              H = max(DE, F);
              if (LOCAL) H = max(H, 0);
              if (TB) tb_push4(tbw[k >> 3], D - E, DE - F, 0, 0);
            }
            if (BAND) {
              const int dd = j - (top + k);
              if (dd < lo || dd > hi) {
                H = NEG;
                E = NEG;
                F = NEG;
              }
            }
            if (LOCAL) m = max(m, H);
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
            for (int w = 0; w < WPS; ++w) tbp[tb_base + ((int64_t)t * WPS + w) * 32 + lane] = tbw[w];
          }
          if (lane == 31 && s + 1 < nstrips) sbuf[j] = make_int2(Hup, Fup);
          // Best cell (local): rows past M never exceed the lane's running best
          // of valid cells (their diagonal scores are -128 and their gap values
          // derive from valid cells minus a gap cost), so the unmasked column
          // max only triggers the masked scan when a valid cell may qualify.
          if (LOCAL && m > 0 && m >= bestv) {
            int mv = 0, ii = INT_MAX;
#pragma unroll
            for (int k = R - 1; k >= 0; --k)
              if (top + k <= M && Hc[k] >= mv && Hc[k] > 0) {
                mv = Hc[k];
                ii = top + k;
              }
            // (mv, ii): the largest valid value and, scanning upward, its smallest row
            if (mv > 0 && (mv > bestv || (mv == bestv && ii < besti))) {
              bestv = mv;
              besti = ii;
              bestj = j;
            }
          }
        }
      }
      if (TB) tb_base += strip_tb_words(jlo, jhi, R);
      if (!LOCAL && s == nstrips - 1 && top <= M && M < top + R) {
#pragma unroll
        for (int k = 0; k < R; ++k)
          if (top + k == M) endH = Hc[k];
      }
      prev_jlo = jlo;
      prev_jhi = jhi;
      __syncwarp();
    }

    // cells evaluated: the band's cells inside the matrix
    uint64_t cells;
    if (BAND) {
      uint64_t c = 0;
      for (int i = lane + 1; i <= M; i += 32) {
        const int a0 = max(1, i + lo), b0 = min(N, i + hi);
        if (b0 >= a0) c += (uint64_t)(b0 - a0 + 1);
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) c += __shfl_down_sync(FULLMASK, c, off);
      cells = c;
    } else {
      cells = (uint64_t)M * (uint64_t)N;
    }
    int score = 0, ei = 0, ej = 0, status = FILTR_ST_OK;
    if (LOCAL) {
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const int ov = __shfl_down_sync(FULLMASK, bestv, off);
        const int oi = __shfl_down_sync(FULLMASK, besti, off);
        const int oj = __shfl_down_sync(FULLMASK, bestj, off);
        if (ov > bestv || (ov == bestv && (oi < besti || (oi == besti && oj < bestj)))) {
          bestv = ov;
          besti = oi;
          bestj = oj;
        }
      }
      if (bestv > 0) {
        score = bestv;
        ei = besti;
        ej = bestj;
      } else {
        status = FILTR_ST_EMPTY;
      }
    } else {
      const int owner = ((M - 1) % HS) / R;
      endH = __shfl_sync(FULLMASK, endH, owner);
      const bool corner_in_band = !BAND || ((N - M) >= lo && (N - M) <= hi);
      if (corner_in_band && endH > NEG_HALF) {
        score = endH;
        ei = M;
        ej = N;
      } else {
        status = FILTR_ST_UNREACHABLE;
        ei = M;
        ej = N;
      }
    }
    if (lane == 0) {
      filtr_result res;
      res.score = score;
      res.q_end = ei;
      res.r_end = ej;
      res.q_begin = (LOCAL && status == FILTR_ST_OK) ? -1 : 0;
      res.r_begin = res.q_begin;
      if (status == FILTR_ST_EMPTY) {
        res.q_end = 0;
        res.r_end = 0;
      }
      res.status = status;
      res.cigar_len = 0;
      res.reserved = 0;
      res.cigar_off = 0;
      res.cells = cells;
      a.out[p] = res;
      FwdOut f;
      f.score = score;
      f.end_i = res.q_end;
      f.end_j = res.r_end;
      f.status = status;
      a.fwd[p] = f;
    }
  }
}

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND>
cudaError_t launch_t(const FullArgs &a, int grid, cudaStream_t s) {
  auto k = k_full<R, LOCAL, AFFINE, TB, BAND>;
  const int smem = full_smem_bytes(R, a.sp.alphabet);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, FULL_WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND>
int occ_t(int smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_full<R, LOCAL, AFFINE, TB, BAND>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_full<R, LOCAL, AFFINE, TB, BAND>,
                                                FULL_WARPS * 32, smem);
  return nb;
}

template <int R>
cudaError_t dispatch_r(const FullArgs &a, int grid, cudaStream_t s) {
  const bool L = a.sp.mode == FILTR_LOCAL, AF = a.sp.affine != 0, T = a.sp.traceback != 0,
             B = a.sp.use_band != 0;
#define FILTR_CASE(l, af, t, b) \
  if (L == l && AF == af && T == t && B == b) return launch_t<R, l, af, t, b>(a, grid, s);
  FILTR_CASE(false, false, false, false)
  FILTR_CASE(false, false, false, true)
  FILTR_CASE(false, false, true, false)
  FILTR_CASE(false, false, true, true)
  FILTR_CASE(false, true, false, false)
  FILTR_CASE(false, true, false, true)
  FILTR_CASE(false, true, true, false)
  FILTR_CASE(false, true, true, true)
  FILTR_CASE(true, false, false, false)
  FILTR_CASE(true, false, false, true)
  FILTR_CASE(true, false, true, false)
  FILTR_CASE(true, false, true, true)
  FILTR_CASE(true, true, false, false)
  FILTR_CASE(true, true, false, true)
  FILTR_CASE(true, true, true, false)
  FILTR_CASE(true, true, true, true)
#undef FILTR_CASE
  return cudaErrorInvalidValue;
}

template <int R>
int occ_r(const ScoreParams &sp, int smem) {
  const bool L = sp.mode == FILTR_LOCAL, AF = sp.affine != 0, T = sp.traceback != 0,
             B = sp.use_band != 0;
#define FILTR_CASE(l, af, t, b) \
  if (L == l && AF == af && T == t && B == b) return occ_t<R, l, af, t, b>(smem);
  FILTR_CASE(false, false, false, false)
  FILTR_CASE(false, false, false, true)
  FILTR_CASE(false, false, true, false)
  FILTR_CASE(false, false, true, true)
  FILTR_CASE(false, true, false, false)
  FILTR_CASE(false, true, false, true)
  FILTR_CASE(false, true, true, false)
  FILTR_CASE(false, true, true, true)
  FILTR_CASE(true, false, false, false)
  FILTR_CASE(true, false, false, true)
  FILTR_CASE(true, false, true, false)
  FILTR_CASE(true, false, true, true)
  FILTR_CASE(true, true, false, false)
  FILTR_CASE(true, true, false, true)
  FILTR_CASE(true, true, true, false)
  FILTR_CASE(true, true, true, true)
#undef FILTR_CASE
  return 0;
}

}  // namespace

int full_smem_bytes(int R, int alphabet) { return 512 + FULL_WARPS * alphabet * 32 * R; }

int full_max_blocks_per_sm(int R, const ScoreParams &sp, int alphabet) {
  const int smem = full_smem_bytes(R, alphabet);
  return R == 8 ? occ_r<8>(sp, smem) : occ_r<16>(sp, smem);
}

cudaError_t launch_full(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (R == 8) return dispatch_r<8>(a, grid, s);
  if (R == 16) return dispatch_r<16>(a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace filtr
