// k_long.cu -- one long pair with every SM on it (full matrix or static band).
//
// The query is cut into row strips of 32*R rows (k_strip.cuh, R = LONG_R).
// All warps of a cooperatively launched grid (so every warp is resident) take
// strips round-robin: warp w handles strips w, w + NW, w + 2NW, ...  Strip s
// needs the bottom row of strip s-1, which is being computed at the same time
// by another warp: lane 31 of strip s-1 writes (H, F) per column into a ring
// slot and, every 16 columns, publishes a 64-bit progress word (strip << 32 |
// column) with a release store (slots are indexed from the strip's first
// column, so a banded pair needs only band-wide slots); lane 0 of strip s
// waits with acquire loads until the column it needs is published, and the
// warp then fetches every published column it can use (up to 32) at once.  A
// ring of NW slots suffices: strip s-1+NW reuses strip s-1's slot, and it
// cannot reach column c before strip s has read column c (the chain s, s+1,
// ..., s-2+NW must each pass c first; a fetch reads a column before its use).
// No cycle of waits exists (every wait is on a smaller strip number), and
// every wait is bounded by a timeout on %globaltimer, after which the kernel
// sets an error flag, every warp stops at its next wait, and the host returns
// FILTR_ERR_TIMEOUT.
#include "k_strip.cuh"

namespace filtr {
namespace {

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct RingIO {
  static constexpr bool FETCH = true;
  int2 *ring;
  uint32_t stride;
  unsigned long long *prog;
  int *err;
  unsigned long long timeout_ns;
  int nw, s, withhold;
  int jlo, prev_jlo, prev_jhi;  // ring slots are indexed from each strip's first column
  int ready;  // columns of strip s-1 known to be published

  __device__ bool wait(int j) {
    if (j <= ready) return true;
    const int lane = threadIdx.x & 31;
    int ok = 1, got = ready;
    if (lane == 0) {
      const unsigned long long want = ((unsigned long long)(s - 1) << 32) | (unsigned)j;
      const unsigned long long *slot = prog + (s - 1) % nw;
      const unsigned long long t0 = gtimer();
      for (;;) {
        const unsigned long long v = ld_acquire(slot);
        if (v >= want) {
          // a later strip in the slot means strip s-1 finished every column
          got = ((v >> 32) == (unsigned long long)(s - 1)) ? (int)(v & 0xffffffffu) : prev_jhi;
          break;
        }
        if (*(volatile int *)err) {
          ok = 0;
          break;
        }
        if (gtimer() - t0 > timeout_ns) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    ok = __shfl_sync(STRIP_FULLMASK, ok, 0);
    ready = __shfl_sync(STRIP_FULLMASK, got, 0);
    return ok != 0;
  }
  __device__ int2 in(int j) { return __ldcg(ring + (size_t)((s - 1) % nw) * stride + (j - prev_jlo)); }
  // After wait(j): the published columns j .. min(ready, jmax, j + 31), lane x
  // loading column j + x.  The warp barrier orders the other lanes' loads after
  // lane 0's acquire.
  __device__ int fetch(int j, int jmax, int2 &v) {
    __syncwarp();
    const int n = min(min(ready, jmax) - j + 1, 32), x = threadIdx.x & 31;
    if (x < n) v = __ldcg(ring + (size_t)((s - 1) % nw) * stride + (j + x - prev_jlo));
    return n;
  }
  __device__ void out(int j, int H, int F) {
    __stcg(ring + (size_t)(s % nw) * stride + (j - jlo), make_int2(H, F));
  }
  // Lane 31 writes the ring and publishes: its release store orders its own
  // ring writes before the progress word, so no separate fence is needed.
  __device__ void done_col(int j, int jlo, int jhi) {
    if ((((j - jlo) & 15) == 15 || j == jhi) && !(withhold && s == 0)) {
      st_release(prog + s % nw, ((unsigned long long)s << 32) | (unsigned)j);
    }
  }
};

template <int R, bool LOCAL, bool AFFINE, bool TB, bool BAND>
__global__ void __launch_bounds__(FULL_WARPS * 32) k_long(const LongArgs a) {
  constexpr int HS = 32 * R;
  extern __shared__ __align__(16) int8_t smem[];
  const int A = a.sp.alphabet;
  int8_t *s_sub = smem;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < A * A; t += blockDim.x) s_sub[t] = a.sp.subst[t];
  __syncthreads();
  const int gw = blockIdx.x * FULL_WARPS + wib;
  const int nw = gridDim.x * FULL_WARPS;

  StripPair P;
  P.M = a.M;
  P.N = a.N;
  P.q = a.q;
  P.r = a.r;
  P.lo = a.lo;
  P.hi = a.hi;
  P.one = (a.sp.alphabet > 0) ? 1 : 0;  // 1, unknown to the compiler
  P.o = a.sp.o;
  P.e = a.sp.e;
  P.A = A;
  P.s_sub = s_sub;
  P.prof = smem + 512 + wib * (A * HS);
  P.tb = a.tb;
  const int M = a.M, N = a.N;
  const int nstrips = (M + HS - 1) / HS;

  RingIO io;
  io.ring = a.ring;
  io.stride = a.ring_stride;
  io.prog = a.prog;
  io.err = a.err;
  io.timeout_ns = a.timeout_ns;
  io.nw = nw;
  io.withhold = a.withhold;
  LaneBest best{0, INT_MAX, INT_MAX};
  int endH = NEG;
  bool had_last = false;
  for (int s = gw; s < nstrips; s += nw) {
    if (*(volatile int *)a.err) break;
    int64_t jl, jh, pjl = 1, pjh = 0;
    strip_cols((int64_t)s * HS, HS, M, N, BAND, a.lo, a.hi, &jl, &jh);
    if (jl > jh) break;
    if (s > 0) strip_cols((int64_t)(s - 1) * HS, HS, M, N, BAND, a.lo, a.hi, &pjl, &pjh);
    io.s = s;
    io.jlo = (int)jl;
    io.prev_jlo = (int)pjl;
    io.prev_jhi = (int)pjh;
    io.ready = 0;
    const int64_t base = TB ? a.strip_base[s] : 0;
    if (!strip_pass<R, LOCAL, AFFINE, TB, BAND>(P, s, (int)jl, (int)jh, (int)pjl, (int)pjh, base, io,
                                                best, endH))
      break;
    if (s == nstrips - 1) had_last = true;
  }
  best = warp_best(best);
  if (had_last) {
    const int owner = ((M - 1) % HS) / R;
    endH = __shfl_sync(STRIP_FULLMASK, endH, owner);
  }
  if (lane == 0) {
    a.wbest[gw] = best;
    if (had_last) *a.end_h = endH;
  }
}

// Reduce the warps' best cells and the corner into the pair's result.
__global__ void k_long_finish(const LongArgs a, int nw, uint64_t cells, filtr_result *out,
                              FwdOut *fwd) {
  __shared__ LaneBest sb[32];
  LaneBest b{0, INT_MAX, INT_MAX};
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const LaneBest o = a.wbest[w];
    if (o.v > b.v || (o.v == b.v && (o.i < b.i || (o.i == b.i && o.j < b.j)))) b = o;
  }
  b = warp_best(b);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    const LaneBest o = sb[w];
    if (o.v > b.v || (o.v == b.v && (o.i < b.i || (o.i == b.i && o.j < b.j)))) b = o;
  }
  filtr_result res{};
  res.cells = cells;
  const bool local = a.sp.mode == FILTR_LOCAL;
  if (*(volatile int *)a.err) {
    res.status = FILTR_ST_TIMEOUT;
    *out = res;
    FwdOut f{0, 0, 0, FILTR_ST_TIMEOUT};
    *fwd = f;
    return;
  }
  if (local) {
    if (b.v > 0) {
      res.score = b.v;
      res.q_end = b.i;
      res.r_end = b.j;
      res.q_begin = res.r_begin = -1;
      res.status = FILTR_ST_OK;
    } else {
      res.status = FILTR_ST_EMPTY;
    }
  } else {
    const int eh = *a.end_h;
    const bool corner = (a.N - a.M) >= a.lo && (a.N - a.M) <= a.hi;
    res.q_end = a.M;
    res.r_end = a.N;
    if (corner && eh > NEG_HALF) {
      res.score = eh;
      res.status = FILTR_ST_OK;
    } else {
      res.status = FILTR_ST_UNREACHABLE;
    }
  }
  *out = res;
  FwdOut f;
  f.score = res.score;
  f.end_i = res.q_end;
  f.end_j = res.r_end;
  f.status = res.status;
  *fwd = f;
}

template <bool LOCAL, bool AFFINE, bool TB, bool BAND>
cudaError_t coop(const LongArgs &a, int grid, cudaStream_t s) {
  constexpr int R = LONG_R;
  auto k = k_long<R, LOCAL, AFFINE, TB, BAND>;
  const int smem = full_smem_bytes(R, a.sp.alphabet);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  LongArgs copy = a;
  void *args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void *)k, grid, FULL_WARPS * 32, args, smem, s);
}

template <bool LOCAL, bool AFFINE, bool TB, bool BAND>
int occ_long() {
  constexpr int R = LONG_R;
  int nb = 0;
  auto k = k_long<R, LOCAL, AFFINE, TB, BAND>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, full_smem_bytes(R, 20));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, FULL_WARPS * 32, full_smem_bytes(R, 20));
  return nb;
}

}  // namespace

int long_blocks_per_sm(const ScoreParams &sp) {
  const bool L = sp.mode == FILTR_LOCAL, AF = sp.affine != 0, T = sp.traceback != 0,
             B = sp.use_band != 0;
#define FILTR_CASE(l, af, t, b) \
  if (L == l && AF == af && T == t && B == b) return occ_long<l, af, t, b>();
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

cudaError_t launch_long(const LongArgs &a, int grid, cudaStream_t s) {
  const bool L = a.sp.mode == FILTR_LOCAL, AF = a.sp.affine != 0, T = a.sp.traceback != 0,
             B = a.sp.use_band != 0;
#define FILTR_CASE(l, af, t, b) \
  if (L == l && AF == af && T == t && B == b) return coop<l, af, t, b>(a, grid, s);
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

cudaError_t launch_long_finish(const LongArgs &a, int nw, uint64_t cells, filtr_result *out,
                               FwdOut *fwd, cudaStream_t s) {
  k_long_finish<<<1, 1024, 0, s>>>(a, nw, cells, out, fwd);
  return cudaGetLastError();
}

}  // namespace filtr
