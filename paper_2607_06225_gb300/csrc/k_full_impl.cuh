// k_full_impl.cuh -- the batched tiled wavefront kernel (template body),
// instantiated for narrow (R = 8, 16) and wide (R = 24, 32) row tiles in two
// translation units that compile in parallel.
//
// One warp aligns one pair at a time, pulling pairs from a work queue over a
// cost-descending order (persistent grid).  The query is cut into strips of
// 32*R rows processed one after another by the same warp (see k_strip.cuh for
// the strip schedule and the cell update); a strip's bottom row goes to a
// per-warp global buffer that the next strip's lane 0 reads back -- lane 0
// reads column j long before lane 31 overwrites it, so one buffer serves both.
#pragma once

#include "k_strip.cuh"
#include "plan.h"

namespace filtr {
namespace {

// Strip I/O through one per-warp buffer (no cross-warp waits).
struct WarpIO {
  int2 *buf;
  __device__ bool wait(int) { return true; }
  static constexpr bool FETCH = false;
  __device__ int2 in(int j) { return buf[j]; }
  __device__ void out(int j, int H, int F) { buf[j] = make_int2(H, F); }
  __device__ void done_col(int, int, int) {}
};

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND, bool GR>
__global__ void __launch_bounds__(FULL_WARPS * 32) k_full(const FullArgs a) {
  constexpr int HS = 32 * R;
  extern __shared__ __align__(16) int8_t smem[];
  if (launch_idle<GR>(a)) return;  // uniform over the block
  const int A = a.sp.alphabet;
  int8_t *s_sub = smem;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < A * A; t += blockDim.x) s_sub[t] = a.sp.subst[t];
  __syncthreads();
  const int gw = blockIdx.x * FULL_WARPS + wib;
  WarpIO io{a.strip_buf + (size_t)gw * a.strip_stride};

  for (;;) {
    uint32_t t0 = 0;
    if (lane == 0) t0 = atomicAdd(a.counter, 1u);
    t0 = __shfl_sync(STRIP_FULLMASK, t0, 0);
    if (t0 >= launch_n<GR>(a)) break;
    const uint32_t *order = launch_order<GR>(a);
    const uint32_t p = order ? order[t0] : t0;
    const BatchDev bv = launch_batch<GR>(a);
    StripPair P;
    P.M = (int)bv.q_len[p];
    P.N = (int)bv.r_len[p];
    P.q = bv.q_seq + bv.q_off[p];
    P.r = bv.r_seq + bv.r_off[p];
    P.lo = -P.M - 1;
    P.hi = P.N + 1;
    if (BAND) {
      int64_t l64, h64;
      band_limits(P.M, P.N, a.sp.band, a.sp.band_literal, &l64, &h64);
      P.lo = (int)(l64 < -(int64_t)P.M - 1 ? -(int64_t)P.M - 1 : l64);
      P.hi = (int)(h64 > (int64_t)P.N + 1 ? (int64_t)P.N + 1 : h64);
    }
    P.one = (a.sp.alphabet > 0) ? 1 : 0;  // 1, unknown to the compiler
    P.o = a.sp.o;
    P.e = a.sp.e;
    P.A = A;
    P.s_sub = s_sub;
    P.prof = smem + 512 + wib * (A * HS);
    P.tb = TB ? a.tb + a.tbl[p].off : nullptr;
    const int M = P.M, N = P.N;
    if ((a.max_n && (uint32_t)N > a.max_n) || (a.max_m && (uint32_t)M > a.max_m)) {
      // only the fixed-scratch entry point sets these limits
      if (lane == 0) {
        filtr_result res{};
        res.status = FILTR_ST_TOO_WIDE;
        launch_out<GR>(a)[p] = res;
      }
      continue;
    }

    const int nstrips = (M + HS - 1) / HS;
    LaneBest best{0, INT_MAX, INT_MAX};
    int endH = NEG;
    int64_t tb_base = 0;
    int prev_jlo = 1, prev_jhi = 0;
    for (int s = 0; s < nstrips; ++s) {
      int64_t jl64, jh64;
      strip_cols((int64_t)s * HS, HS, M, N, BAND, P.lo, P.hi, &jl64, &jh64);
      const int jlo = (int)jl64, jhi = (int)jh64;
      if (jlo > jhi) break;  // no band cell in this strip or below
      strip_pass<R, LOCAL, AFFINE, TB, BAND>(P, s, jlo, jhi, prev_jlo, prev_jhi, tb_base, io, best,
                                             endH);
      if (TB) tb_base += strip_tb_words(jlo, jhi, R);
      prev_jlo = jlo;
      prev_jhi = jhi;
    }

    // cells evaluated: the band's cells inside the matrix
    uint64_t cells;
    if (BAND) {
      uint64_t c = 0;
      for (int i = lane + 1; i <= M; i += 32) {
        const int a0 = max(1, i + P.lo), b0 = min(N, i + P.hi);
        if (b0 >= a0) c += (uint64_t)(b0 - a0 + 1);
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) c += __shfl_down_sync(STRIP_FULLMASK, c, off);
      cells = c;
    } else {
      cells = (uint64_t)M * (uint64_t)N;
    }
    int score = 0, ei = 0, ej = 0, status = FILTR_ST_OK;
    if (LOCAL) {
      best = warp_best(best);
      if (best.v > 0) {
        score = best.v;
        ei = best.i;
        ej = best.j;
      } else {
        status = FILTR_ST_EMPTY;
      }
    } else {
      const int owner = ((M - 1) % HS) / R;
      endH = __shfl_sync(STRIP_FULLMASK, endH, owner);
      const bool corner_in_band = !BAND || ((N - M) >= P.lo && (N - M) <= P.hi);
      ei = M;
      ej = N;
      if (corner_in_band && endH > NEG_HALF)
        score = endH;
      else
        status = FILTR_ST_UNREACHABLE;
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
      launch_out<GR>(a)[p] = res;
      if (a.fwd) {
        FwdOut f;
        f.score = score;
        f.end_i = res.q_end;
        f.end_j = res.r_end;
        f.status = status;
        a.fwd[p] = f;
      }
    }
  }
}

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND, bool GR>
cudaError_t launch_t(const FullArgs &a, int grid, cudaStream_t s) {
  auto k = k_full<R, LOCAL, AFFINE, TB, BAND, GR>;
  const int smem = full_smem_bytes(R, a.sp.alphabet);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, FULL_WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND, bool GR>
int occ_t(int smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_full<R, LOCAL, AFFINE, TB, BAND, GR>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_full<R, LOCAL, AFFINE, TB, BAND, GR>,
                                                FULL_WARPS * 32, smem);
  return nb;
}

#define FILTR_FULL_CASES(X) \
  X(false, false, false, false) \
  X(false, false, false, true)  \
  X(false, false, true, false)  \
  X(false, false, true, true)   \
  X(false, true, false, false)  \
  X(false, true, false, true)   \
  X(false, true, true, false)   \
  X(false, true, true, true)    \
  X(true, false, false, false)  \
  X(true, false, false, true)   \
  X(true, false, true, false)   \
  X(true, false, true, true)    \
  X(true, true, false, false)   \
  X(true, true, false, true)    \
  X(true, true, true, false)    \
  X(true, true, true, true)

template <int R, bool GR>
cudaError_t dispatch_r(const FullArgs &a, int grid, cudaStream_t s) {
  const bool L = a.sp.mode == FILTR_LOCAL, AF = a.sp.affine != 0, T = a.sp.traceback != 0,
             B = a.sp.use_band != 0;
#define FILTR_CASE(l, af, t, b) \
  if (L == l && AF == af && T == t && B == b) return launch_t<R, l, af, t, b, GR>(a, grid, s);
  FILTR_FULL_CASES(FILTR_CASE)
#undef FILTR_CASE
  return cudaErrorInvalidValue;
}

template <int R, bool GR>
int occ_r(const ScoreParams &sp, int smem) {
  const bool L = sp.mode == FILTR_LOCAL, AF = sp.affine != 0, T = sp.traceback != 0,
             B = sp.use_band != 0;
#define FILTR_CASE(l, af, t, b) \
  if (L == l && AF == af && T == t && B == b) return occ_t<R, l, af, t, b, GR>(smem);
  FILTR_FULL_CASES(FILTR_CASE)
#undef FILTR_CASE
  return 0;
}

}  // namespace
}  // namespace filtr
