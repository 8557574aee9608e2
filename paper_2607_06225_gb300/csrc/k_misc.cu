// k_misc.cu -- small kernels: empty-sequence pairs, residue validation and
// packing, and the integer / DPX throughput probe used as the roofline
// denominator of the cell update.
#include "filtr_internal.h"
#include "plan.h"

namespace filtr {
namespace {

// Pairs with M == 0 or N == 0 evaluate no cell.  Global: the only alignment is
// one gap of max(M, N) (score -(o + L*e), 0 if both are empty); local: empty.
__global__ void k_trivial(const BatchDev b0, const ScoreParams sp, const uint32_t *order, uint32_t n,
                          filtr_result *out, FwdOut *fwd, const GraphDesc *gd,
                          const DevPlanSummary *gsum) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  BatchDev b = b0;
  if (gd) {  // captured pipeline: the empty pairs follow every shape's slice
    if (gd->abort) return;
    b = gd->b;
    out = gd->out;
    uint32_t begin = 0;
    for (int k = 0; k < SHAPE_TILED; ++k) begin += gsum->count[k];
    order += begin;
    n = gsum->count[KEY_TRIVIAL];
  }
  if (t >= n) return;
  const uint32_t p = order[t];
  const int M = (int)b.q_len[p], N = (int)b.r_len[p];
  filtr_result r;
  r.cigar_len = 0;
  r.reserved = 0;
  r.cigar_off = 0;
  r.cells = 0;
  r.q_begin = 0;
  r.r_begin = 0;
  FwdOut f;
  if (sp.mode == FILTR_LOCAL) {
    r.score = 0;
    r.q_end = 0;
    r.r_end = 0;
    r.status = FILTR_ST_EMPTY;
  } else {
    const int L = M > N ? M : N;
    r.score = (L == 0) ? 0 : -(sp.o + L * sp.e);
    r.q_end = M;
    r.r_end = N;
    r.status = FILTR_ST_OK;
    if (sp.use_band && sp.band_literal && (N - M > sp.band || M - N > sp.band)) {
      r.score = 0;  // the literal band misses the corner
      r.status = FILTR_ST_UNREACHABLE;
    }
  }
  f.score = r.score;
  f.end_i = r.q_end;
  f.end_j = r.r_end;
  f.status = r.status;
  out[p] = r;
  fwd[p] = f;
}

__global__ void k_validate(const uint8_t *codes, uint64_t n, int alphabet, uint32_t *bad) {
  uint32_t cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t * 16 < n; t += stride) {
    const uint64_t base = t * 16;
    if (base + 16 <= n && (reinterpret_cast<uintptr_t>(codes + base) & 15) == 0) {
      const uint4 v = *reinterpret_cast<const uint4 *>(codes + base);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 16; ++k) cnt += ((w[k >> 2] >> (8 * (k & 3))) & 0xff) >= (uint32_t)alphabet;
    } else {
      for (uint64_t x = base; x < base + 16 && x < n; ++x) cnt += codes[x] >= alphabet;
    }
  }
  for (int off = 16; off; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

// One warp per pair: count residue codes >= alphabet in q and r.
__global__ void k_validate_pairs(const BatchDev b0, uint32_t n, int alphabet, uint32_t *bad,
                                 const GraphDesc *gd) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const BatchDev b = gd ? gd->b : b0;  // captured pipeline: batch and count from gd
  if (gd) n = gd->n;
  if (w >= n) return;
  uint32_t cnt = 0;
  const uint8_t *q = b.q_seq + b.q_off[w];
  const uint8_t *r = b.r_seq + b.r_off[w];
  const uint32_t M = b.q_len[w], N = b.r_len[w];
  for (uint32_t x = lane; x < M; x += 32) cnt += q[x] >= alphabet;
  for (uint32_t x = lane; x < N; x += 32) cnt += r[x] >= alphabet;
  for (int off = 16; off; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
  if (lane == 0 && cnt) atomicAdd(bad, cnt);
}

// DNA: 16 codes of 2 bits per word; protein: 4 codes of 8 bits per word.
// 16 codes per thread from one 16-byte load: DNA packs them into one word
// (2 bits each), protein copies them as four words (8 bits each); codes at or
// above the alphabet are counted.  `codes` must be 16-byte aligned; the last
// partial group of 16 is read byte by byte.
__global__ void k_pack(const uint8_t *codes, uint64_t n, int alphabet, uint32_t *packed,
                       uint32_t *bad) {
  const bool dna = alphabet <= 4;
  const uint32_t lim = (uint32_t)alphabet - 1u;
  const uint32_t limv = lim * 0x01010101u;
  const uint64_t groups = (n + 15) / 16;
  uint32_t cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < groups; g += stride) {
    uint32_t x[4];
    if (g * 16 + 16 <= n) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(codes) + g);
      x[0] = v.x;
      x[1] = v.y;
      x[2] = v.z;
      x[3] = v.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) cnt += __popc(__vcmpgtu4(x[k], limv)) >> 3;
    } else {  // the tail: bytes past n count as code 0
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t w = 0;
        for (int b = 0; b < 4; ++b) {
          const uint64_t t = g * 16 + 4 * k + b;
          const uint32_t c = t < n ? codes[t] : 0u;
          cnt += c > lim;
          w |= (c & 0xffu) << (8 * b);
        }
        x[k] = w;
      }
    }
    if (dna) {  // four bytes -> 8 bits: code b at bits 2b
      uint32_t out = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t t = x[k] & 0x03030303u;
        t = (t | (t >> 6)) & 0x000f000fu;
        t = (t | (t >> 12)) & 0xffu;
        out |= t << (8 * k);
      }
      packed[g] = out;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (g * 4 + k < (n + 3) / 4) packed[g * 4 + k] = x[k];
    }
  }
  for (int off = 16; off; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

// ---- throughput probe ---------------------------------------------------------
// Each thread runs CH independent dependency chains of one operation for ITERS
// iterations; the result is folded into a store that depends on every chain so
// nothing is dead code.  kind 0: x = max(x + a, y) written as two plain int32
// ops (counted as 2 ops); 1: __viaddmax_s32; 2: __vimax3_s32; 3: __viaddmax_s16x2.
constexpr int CH = 8;

template <int KIND>
__global__ void k_probe(int iters, int seed, int *sink, long long *clk, unsigned long long *ns) {
  int x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = seed + c * 7 + threadIdx.x;
  const int a = seed & 3, y = seed - 5;
  long long c0 = 0;
  unsigned long long t0 = 0;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (KIND == 0) {
        x[c] = max(x[c] + a, y + c);
      } else if (KIND == 1) {
        x[c] = __viaddmax_s32(x[c], a, y + c);
      } else if (KIND == 2) {
        x[c] = __vimax3_s32(x[c], y + c, x[(c + 1) % CH] - 1);
      } else {
        x[c] = (int)__viaddmax_s16x2((unsigned)x[c], (unsigned)a, (unsigned)(y + c));
      }
    }
  }
  int acc = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) acc ^= x[c];
  if (acc == 0x7fffffff) sink[blockIdx.x] = acc;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    *clk = clock64() - c0;
    *ns = t1 - t0;
  }
}

template <int KIND>
double probe_one(int sms, int *sink, long long *clk, unsigned long long *ns, double *hz) {
  const int threads = 512, blocks = sms * 4, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe<KIND><<<blocks, threads>>>(64, 3, sink, clk, ns);  // warm-up
  cudaEventRecord(e0);
  k_probe<KIND><<<blocks, threads>>>(iters, 3, sink, clk, ns);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  long long hc = 0;
  unsigned long long hn = 0;
  cudaMemcpy(&hc, clk, sizeof hc, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hn, ns, sizeof hn, cudaMemcpyDeviceToHost);
  if (hn > 0) *hz = (double)hc / ((double)hn * 1e-9);
  const double ops = (double)blocks * threads * iters * CH * (KIND == 0 ? 2.0 : 1.0);
  return ops / (ms * 1e-3);
}

}  // namespace

cudaError_t launch_trivial(const BatchDev &b, const ScoreParams &sp, const uint32_t *order,
                           uint32_t n, filtr_result *out, FwdOut *fwd, cudaStream_t s,
                           const GraphDesc *gd, const DevPlanSummary *gsum) {
  if (n == 0) return cudaSuccess;
  k_trivial<<<(n + 127) / 128, 128, 0, s>>>(b, sp, order, n, out, fwd, gd, gsum);
  return cudaGetLastError();
}

cudaError_t launch_validate(const uint8_t *codes, uint64_t n, int alphabet, uint32_t *bad,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  uint64_t chunks = (n + 15) / 16;
  unsigned blocks = (unsigned)((chunks + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_validate<<<blocks, 256, 0, s>>>(codes, n, alphabet, bad);
  return cudaGetLastError();
}

cudaError_t launch_validate_pairs(const BatchDev &b, uint32_t n, int alphabet, uint32_t *bad,
                                  cudaStream_t s, const GraphDesc *gd) {
  if (n == 0) return cudaSuccess;
  const uint64_t threads = (uint64_t)n * 32;
  k_validate_pairs<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(b, n, alphabet, bad, gd);
  return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *codes, uint64_t n, int alphabet, uint32_t *packed,
                        uint32_t *bad, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t groups = (n + 15) / 16;
  unsigned blocks = (unsigned)((groups + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_pack<<<blocks, 256, 0, s>>>(codes, n, alphabet, packed, bad);
  return cudaGetLastError();
}

cudaError_t run_probe(double out[5]) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int *sink = nullptr;
  long long *clk = nullptr;
  unsigned long long *ns = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(int) * sms * 4 + 64);
  if (e != cudaSuccess) return e;
  clk = reinterpret_cast<long long *>(reinterpret_cast<char *>(sink) + ((sizeof(int) * sms * 4 + 15) / 16) * 16);
  ns = reinterpret_cast<unsigned long long *>(clk + 1);
  double hz = 0;
  out[0] = probe_one<0>(sms, sink, clk, ns, &hz);
  out[1] = probe_one<1>(sms, sink, clk, ns, &hz);
  out[2] = probe_one<2>(sms, sink, clk, ns, &hz);
  out[3] = probe_one<3>(sms, sink, clk, ns, &hz) * 2.0;  // two 16-bit lanes per op
  out[4] = hz;
  e = cudaGetLastError();
  cudaFree(sink);
  return e;
}

}  // namespace filtr
