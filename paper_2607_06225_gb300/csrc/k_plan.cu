// k_plan.cu -- the batch planner on the device (declared in plan.h).
//
// The host planner walks every pair on one core (shape choice, cost bucket,
// counting sort, traceback layout); for a large tiled batch that is several
// milliseconds during which the GPU waits.  These three launches build the same
// plan from the lengths already in device memory in a few microseconds, and
// their totals come back to the host with the validation count in the one copy
// the call makes before its forward launches.
#include "plan.h"

namespace filtr {
namespace {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Exclusive prefix sum over the block (NT threads, every thread calls it);
// *total receives the block's sum.
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long *ws,
                                                              unsigned long long *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = lane < NT / 32 ? ws[lane] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL_MASK, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) ws[lane] = t;
  }
  __syncthreads();
  const unsigned long long before = w ? ws[w - 1] : 0ull;
  *total = ws[NT / 32 - 1];
  __syncthreads();  // ws is reused by the next call
  return before + x - v;
}

// The pair count and lengths of this launch (a captured pipeline's come from
// its descriptor; its grids are sized for the graph's capacity).
struct PlanView {
  uint32_t n;
  const uint32_t *q_len, *r_len;
};
__device__ __forceinline__ PlanView plan_view(const DevPlanArgs &a) {
  if (a.gd) return PlanView{a.gd->n, a.gd->b.q_len, a.gd->b.r_len};
  return PlanView{a.n, a.q_len, a.r_len};
}

// Shape, cost bucket and traceback words of each pair; block histogram of the
// keys; batch totals; staging words per block.
__global__ void __launch_bounds__(DEV_PLAN_BLOCK) k_plan_classify(const DevPlanArgs a) {
  const PlanView V = plan_view(a);
  if (blockIdx.x * DEV_PLAN_BLOCK >= V.n) return;  // uniform over the block
  __shared__ uint32_t hist[PLAN_KEYS];
  __shared__ unsigned long long part[5][DEV_PLAN_BLOCK / 32];
  __shared__ uint32_t pmax[2][DEV_PLAN_BLOCK / 32];
  for (int i = threadIdx.x; i < PLAN_KEYS; i += DEV_PLAN_BLOCK) hist[i] = 0;
  __syncthreads();
  const uint32_t p = blockIdx.x * DEV_PLAN_BLOCK + threadIdx.x;
  // traceback words, cells, staging words, M + N, cells of int16x2 shapes
  unsigned long long v[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
  uint32_t mm = 0, mn = 0;
  if (p < V.n) {
    const uint32_t M = V.q_len[p], N = V.r_len[p];
    mm = M;
    mn = N;
    v[3] = (unsigned long long)M + N;
    v[2] = a.sp.traceback ? v[3] + 1 : 0ull;
    int key = KEY_TRIVIAL * 64;
    uint64_t w = 0;
    if (M != 0 && N != 0) {
      const uint64_t cost = band_cells(M, N, a.sp);
      const int k = choose_shape(a.tab, a.sp, M, N);
      if (a.sp.traceback) w = shape_tb_words(a.tab, k, M, N, a.sp);
      v[1] = cost;
      v[4] = a.tab.packed[k] ? cost : 0ull;
      key = k * 64 + cost_bucket_desc(cost);
    }
    v[0] = w;
    a.key[p] = (uint16_t)key;
    a.words[p] = w;
    atomicAdd(&hist[key], 1u);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    unsigned long long x = v[i];
    for (int o = 16; o; o >>= 1) x += __shfl_down_sync(FULL_MASK, x, o);
    if (lane == 0) part[i][wp] = x;
  }
  mm = __reduce_max_sync(FULL_MASK, mm);
  mn = __reduce_max_sync(FULL_MASK, mn);
  if (lane == 0) {
    pmax[0][wp] = mm;
    pmax[1][wp] = mn;
  }
  __syncthreads();
  DevPlanSummary &S = a.state->sum;
  if (threadIdx.x < 5) {
    unsigned long long x = 0;
    for (int k = 0; k < DEV_PLAN_BLOCK / 32; ++k) x += part[threadIdx.x][k];
    if (threadIdx.x == 2) a.blk[blockIdx.x] = x;
    unsigned long long *dst = threadIdx.x == 0   ? &S.tb_words
                              : threadIdx.x == 1 ? &S.cells
                              : threadIdx.x == 2 ? &S.stage_words
                              : threadIdx.x == 3 ? &S.cigar_upper
                                                 : &S.cells_packed;
    if (x) atomicAdd(dst, x);
  } else if (threadIdx.x < 7) {
    const int t = threadIdx.x - 5;
    uint32_t x = 0;
    for (int k = 0; k < DEV_PLAN_BLOCK / 32; ++k) x = max(x, pmax[t][k]);
    atomicMax(t ? &S.max_n : &S.max_m, x);
  }
  for (int i = threadIdx.x; i < PLAN_KEYS; i += DEV_PLAN_BLOCK)
    if (hist[i]) atomicAdd(&a.state->hist[i], hist[i]);
}

// One block: key histogram -> first slot of each (shape, bucket) cell in the
// order (shape-major, most expensive bucket first); pairs per shape; staging
// words per block -> the block's first staging word.
__global__ void __launch_bounds__(1024) k_plan_scan(const DevPlanArgs a, uint32_t nblk) {
  __shared__ unsigned long long ws[32];
  DevPlanState *S = a.state;
  if (a.gd) nblk = (a.gd->n + DEV_PLAN_BLOCK - 1) / DEV_PLAN_BLOCK;
  const uint32_t t = threadIdx.x;
  unsigned long long tot;
  unsigned long long kcarry = 0;
  for (uint32_t base = 0; base < (uint32_t)PLAN_KEYS; base += 1024) {
    const uint32_t i = base + t;
    const unsigned long long h = i < (uint32_t)PLAN_KEYS ? S->hist[i] : 0ull;
    const unsigned long long ex = block_excl_scan<1024>(h, ws, &tot);
    if (i < (uint32_t)PLAN_KEYS) S->cursor[i] = (uint32_t)(kcarry + ex);
    kcarry += tot;
  }
  if (t <= KEY_TRIVIAL) {
    uint32_t c = 0;
    for (int b = 0; b < 64; ++b) c += S->hist[t * 64 + b];
    S->sum.count[t] = c;
  }
  unsigned long long carry = 0;
  for (uint32_t base = 0; base < nblk; base += 1024) {
    const uint32_t i = base + t;
    const unsigned long long x = i < nblk ? a.blk[i] : 0ull;
    const unsigned long long e = block_excl_scan<1024>(x, ws, &tot);
    if (i < nblk) a.blk[i] = carry + e;
    carry += tot;
  }
}

// Scatter: pair ids into their cells (lanes with the same key take their
// slots with one atomic), traceback areas (one atomic per warp), per-pair
// layouts and staging offsets.
__global__ void __launch_bounds__(DEV_PLAN_BLOCK) k_plan_place(const DevPlanArgs a) {
  __shared__ unsigned long long ws[DEV_PLAN_BLOCK / 32];
  const PlanView V = plan_view(a);
  if (blockIdx.x * DEV_PLAN_BLOCK >= V.n) return;  // uniform over the block
  const uint32_t p = blockIdx.x * DEV_PLAN_BLOCK + threadIdx.x;
  const bool valid = p < V.n;
  const int lane = threadIdx.x & 31;
  uint32_t key = 0xffffu;
  unsigned long long w = 0, sw = 0;
  if (valid) {
    key = a.key[p];
    w = a.words[p];
    if (a.sp.traceback) sw = (unsigned long long)V.q_len[p] + V.r_len[p] + 1;
  }
  unsigned long long tot;
  const unsigned long long sx = block_excl_scan<DEV_PLAN_BLOCK>(sw, ws, &tot);

  const uint32_t same = __match_any_sync(FULL_MASK, key);
  const int leader = __ffs(same) - 1;
  uint32_t base = 0;
  if (lane == leader && valid) base = atomicAdd(&a.state->cursor[key], (uint32_t)__popc(same));
  base = __shfl_sync(FULL_MASK, base, leader);
  const uint32_t slot = base + (uint32_t)__popc(same & ((1u << lane) - 1u));

  unsigned long long x = w;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  unsigned long long wbase = 0;
  if (lane == 31 && x) wbase = atomicAdd(&a.state->tb_cursor, x);
  wbase = __shfl_sync(FULL_MASK, wbase, 31);

  if (!valid) return;
  a.order[slot] = p;
  TbLayout L{};
  if (key < (uint32_t)KEY_TRIVIAL * 64) {
    const int k = (int)(key >> 6);
    L.off = wbase + x - w;
    L.family = a.tab.packed[k] ? FAM_PACK : FAM_FULL;
    L.R = (uint8_t)a.tab.R[k];
    L.warps = 1;
    L.valid = a.sp.traceback ? 1 : 0;
  }
  a.tbl[p] = L;
  if (a.sp.traceback) a.stage_off[p] = a.blk[blockIdx.x] + sx;
}

}  // namespace

cudaError_t launch_plan(const DevPlanArgs &a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const uint32_t nblk = (a.n + DEV_PLAN_BLOCK - 1) / DEV_PLAN_BLOCK;
  k_plan_classify<<<nblk, DEV_PLAN_BLOCK, 0, st>>>(a);
  k_plan_scan<<<1, 1024, 0, st>>>(a, nblk);
  k_plan_place<<<nblk, DEV_PLAN_BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace filtr
