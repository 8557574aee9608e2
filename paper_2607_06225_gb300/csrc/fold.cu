// fold.cu -- Nussinov RNA folding (Table 1) with X-drop transferred to it
// (Sec. 9.5): the kernel and the filtr_fold_batch entry point.
//
// One CTA per sequence.  The triangle 0 <= i <= j < n is swept along the span
// k = j - i: the cells of one span depend only on shorter spans, so the CTA's
// threads take a span's positions i in parallel and a barrier separates spans.
// The table lives in global memory span-major (row k holds F(i, i+k) for
// i = 0..n-1-k), so both operand streams of the split term
// max_m F(i,m) + F(m+1,j) -- row t at position i and row k-1-t at position
// i+t+1 -- are contiguous across the threads of a warp for each t.  Pruned and
// unevaluated cells hold NEG.  X-drop (after the warm-up spans) prunes a cell
// when F < best(k-1) - X; the next span's domain is [lo - 1, hi] of the
// unpruned positions; the per-span maximum and bounds come from one block
// reduction.  Thread 0 then walks the fold with a stack in shared memory,
// taking at each cell the first of (i unpaired), (j unpaired), (i pairs j),
// (split at the smallest m) that gives F(i, j).
#include <algorithm>
#include <climits>
#include <vector>

#include "filtr_ctx.h"

namespace filtr {
namespace {

constexpr int FOLD_THREADS = 256;

struct FoldArgs {
  const uint8_t *seq;
  const uint64_t *off;
  const uint32_t *len;
  const uint32_t *order;       // sequences of this launch
  const uint64_t *table_off;   // per sequence (indexed by sequence id): first word of its table
  int32_t *table;
  filtr_fold_result *out;
  int32_t *partner;            // nullptr without traceback
  int min_loop, use_xdrop, xdrop, warmup;
  int max_group;               // largest thread group per cell (1 or 32)
};

__device__ __forceinline__ bool rna_pair(int a, int b) {
  const int s = a + b;  // A=0 C=1 G=2 U=3: A-U and C-G sum to 3, G-U to 5
  return s == 3 || (s == 5 && a != b);
}

// first word of span k's row in a table of n positions
__device__ __forceinline__ int64_t row_off(int k, int n) {
  return (int64_t)k * n - (int64_t)k * (k - 1) / 2;
}

__global__ void __launch_bounds__(FOLD_THREADS) k_fold(const FoldArgs a) {
  __shared__ uint8_t sx[FILTR_FOLD_MAX_LEN];
  __shared__ int red[3][FOLD_THREADS / 32];
  __shared__ unsigned long long redk[FOLD_THREADS / 32];
  __shared__ int16_t stack[2 * FILTR_FOLD_MAX_LEN + 4];  // positions < 4096
  __shared__ int32_t roff[FILTR_FOLD_MAX_LEN];             // row_off(k, n) for every span
  const uint32_t p = a.order[blockIdx.x];
  const int n = (int)a.len[p];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint8_t *g = a.seq + a.off[p];
  for (int t = tid; t < n; t += FOLD_THREADS) sx[t] = g[t];
  int32_t *D = a.table + a.table_off[p];
  for (int t = tid; t < n; t += FOLD_THREADS) D[t] = 0;  // span 0
  for (int t = tid; t < n; t += FOLD_THREADS) roff[t] = (int32_t)row_off(t, n);
  if (a.partner)
    for (int t = tid; t < n; t += FOLD_THREADS) a.partner[a.off[p] + t] = -1;
  __syncthreads();

  int lo = 0, hi = n - 1, best = 0, last_k = 0;
  uint64_t cells = (uint64_t)n;
  for (int k = 1; k < n; ++k) {
    const int dl = max(lo - 1, 0), dh = min(hi, n - 1 - k);
    if (dl > dh) break;
    const int32_t *r1 = D + row_off(k - 1, n);
    const int32_t *r2 = k >= 2 ? D + row_off(k - 2, n) : nullptr;
    int32_t *rk = D + row_off(k, n);
    int tmax = INT_MIN, tlo = INT_MAX, thi = INT_MIN;
    // a group of G threads per cell (G = 1..32, a power of two, as many as the
    // span's domain leaves room for): the group splits the cell's split terms
    // and reduces them with shuffles, so the long, narrow spans near the top of
    // the triangle keep the CTA busy.  The group's lanes read different rows, so
    // this pays only while the resident tables stay in L2 (short sequences)
    int G = 1;
    while (G < a.max_group && 2 * G * (dh - dl + 1) <= FOLD_THREADS) G *= 2;
    const int per_pass = FOLD_THREADS / G, sub = tid & (G - 1), slot = tid / G;
    for (int i0 = 0; i0 <= n - 1 - k; i0 += per_pass) {  // uniform trip count
      const int i = i0 + slot;
      const bool in_dom = i >= dl && i <= dh;
      int f = NEG;
      if (in_dom) {
        const int j = i + k;
        if (sub == 0) {
          f = max(r1[i + 1], r1[i]);  // i unpaired, j unpaired
          if (rna_pair(sx[i], sx[j]) && k - 1 >= a.min_loop) {
            const int inner = k >= 2 ? r2[i + 1] : 0;  // an empty interval is 0
            f = max(f, inner + 1);
          }
        }
        // F(i, i+t) + F(i+t+1, j): o1 -> F(i, i+t) in row t, o2 -> F(i+t+1, j)
        // in row k-1-t, both stepped by whole rows (row t holds n - t cells)
        if (G == 1) {
          int o1 = i, o2 = roff[k - 1] + i + 1;
#pragma unroll 4
          for (int t = 0; t < k; ++t) {
            f = max(f, D[o1] + D[o2]);
            o1 += n - t;
            o2 -= n - k + 1 + t;
          }
        } else if (sub < k) {  // t = sub, sub + G, ...: row_off(a + G) - row_off(a) = G n - G a - G(G-1)/2
          const int gg = G * (G - 1) / 2;
          int o1 = roff[sub] + i, o2 = roff[k - 1 - sub] + i + sub + 1;
          for (int t = sub; t < k; t += G) {
            f = max(f, D[o1] + D[o2]);
            o1 += G * n - G * t - gg;
            o2 -= G * n - G * (k - 1 - t - G) - gg - G;
          }
        }
      }
      for (int o = G >> 1; o; o >>= 1) f = max(f, __shfl_xor_sync(0xffffffffu, f, o));
      if (in_dom) {
        const bool alive = f > NEG_HALF && (!a.use_xdrop || k <= a.warmup || f >= best - a.xdrop);
        if (!alive) f = NEG;
        if (alive) {
          tmax = max(tmax, f);
          tlo = min(tlo, i);
          thi = max(thi, i);
        }
      }
      if (sub == 0 && i <= n - 1 - k) rk[i] = f;
    }
    tmax = __reduce_max_sync(0xffffffffu, tmax);
    tlo = __reduce_min_sync(0xffffffffu, tlo);
    thi = __reduce_max_sync(0xffffffffu, thi);
    if (lane == 0) {
      red[0][wid] = tmax;
      red[1][wid] = tlo;
      red[2][wid] = thi;
    }
    __syncthreads();  // also publishes row k to the whole CTA
    int gmax = INT_MIN, glo = INT_MAX, ghi = INT_MIN;
    for (int w = 0; w < FOLD_THREADS / 32; ++w) {
      gmax = max(gmax, red[0][w]);
      glo = min(glo, red[1][w]);
      ghi = max(ghi, red[2][w]);
    }
    cells += (uint64_t)(dh - dl + 1);
    last_k = k;
    __syncthreads();  // red[] is reused by the next span
    if (glo == INT_MAX) break;  // nothing unpruned on span k
    best = gmax;
    lo = glo;
    hi = ghi;
  }

  // the end cell: (0, n-1) if it stayed, else the best unpruned cell (largest F,
  // then longest span, then smallest i)
  int ei = 0, ej = n - 1, status = FILTR_ST_OK, score = 0;
  if (n > 0) {
    const bool whole = (n - 1 <= last_k) && D[row_off(n - 1, n)] > NEG_HALF;
    if (!whole) {
      unsigned long long key = 0;
      for (int k = 0; k <= last_k; ++k)
        for (int i = tid; i <= n - 1 - k; i += FOLD_THREADS) {
          const int f = D[row_off(k, n) + i];
          if (f > NEG_HALF) {
            const unsigned long long kk = ((unsigned long long)(f + 1) << 40) |
                                          ((unsigned long long)k << 20) |
                                          (unsigned long long)(0xfffff - i);
            key = max(key, kk);
          }
        }
      for (int o = 16; o; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
      if (lane == 0) redk[wid] = key;
      __syncthreads();
      key = 0;
      for (int w = 0; w < FOLD_THREADS / 32; ++w) key = max(key, redk[w]);
      const int k = (int)((key >> 20) & 0xfffff);
      ei = 0xfffff - (int)(key & 0xfffff);
      ej = ei + k;
      status = FILTR_ST_DROPPED;
    }
    score = D[row_off(ej - ei, n) + ei];
  }
  if (tid == 0) {
    filtr_fold_result r;
    r.score = n > 0 ? score : 0;
    r.i_end = ei;
    r.j_end = n > 0 ? ej : 0;
    r.status = status;
    r.cells = cells;
    a.out[p] = r;
  }
  if (!a.partner || n == 0 || tid != 0) return;

  // the fold below the end cell
  int32_t *pt = a.partner + a.off[p];
  int top = 0;
  stack[top++] = (int16_t)ei;
  stack[top++] = (int16_t)ej;
  while (top > 0) {
    const int j = stack[--top], i = stack[--top];
    if (i >= j) continue;
    const int k = j - i;
    const int f = D[row_off(k, n) + i];
    const int32_t *r1 = D + row_off(k - 1, n);
    if (r1[i + 1] == f) {
      stack[top++] = (int16_t)(i + 1);
      stack[top++] = (int16_t)j;
    } else if (r1[i] == f) {
      stack[top++] = (int16_t)i;
      stack[top++] = (int16_t)(j - 1);
    } else if (rna_pair(sx[i], sx[j]) && k - 1 >= a.min_loop &&
               (k >= 2 ? D[row_off(k - 2, n) + i + 1] : 0) + 1 == f) {
      pt[i] = j;
      pt[j] = i;
      stack[top++] = (int16_t)(i + 1);
      stack[top++] = (int16_t)(j - 1);
    } else {
      int t = 0;
      for (; t < k; ++t) {
        const int x = D[row_off(t, n) + i], y = D[row_off(k - 1 - t, n) + i + t + 1];
        if (x > NEG_HALF && y > NEG_HALF && x + y == f) break;
      }
      if (t == k) break;  // no term gives F(i, j): not expected
      stack[top++] = (int16_t)i;
      stack[top++] = (int16_t)(i + t);
      stack[top++] = (int16_t)(i + t + 1);
      stack[top++] = (int16_t)j;
    }
  }
}

struct Carve {
  char *base;
  size_t cap, used = 0;
  template <class T>
  T *take(size_t count, size_t align = 256) {
    used = (used + align - 1) / align * align;
    T *p = reinterpret_cast<T *>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

}  // namespace

static filtr_status fold_impl(Ctx *ctx, const filtr_fold_params *prm, uint32_t n,
                              const uint8_t *seq, const uint64_t *off, const uint32_t *len,
                              filtr_fold_result *out, int32_t *partner, cudaStream_t st) {
  if (!prm) {
    set_error("params is NULL");
    return FILTR_ERR_INVALID;
  }
  if (prm->min_loop < 0 || prm->warmup < 0 || (prm->use_xdrop && prm->xdrop < 0) ||
      (prm->traceback != 0 && prm->traceback != 1)) {
    set_error("fold params: min_loop, warmup and xdrop must be >= 0, traceback 0 or 1");
    return FILTR_ERR_INVALID;
  }
  if (n == 0) return FILTR_OK;
  if (!seq || !off || !len || !out || (prm->traceback && !partner)) {
    set_error("a batch pointer is NULL");
    return FILTR_ERR_INVALID;
  }
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
  if (ctx->done_ev) {
    ce = cudaEventSynchronize(ctx->done_ev);
    if (ce != cudaSuccess) return cuda_fail(ce, "waiting for the previous call");
  }
  ctx->ev_used = 0;
  ctx->spans.clear();
  uint32_t launches = 0;
  // codes (every one below 4) and lengths, one synchronisation
  if (!ctx->ensure_host((size_t)n * 4 + 256)) {
    set_error("pinned host allocation failed");
    return FILTR_ERR_NOMEM;
  }
  uint32_t *h_len = reinterpret_cast<uint32_t *>(ctx->h_stage);
  uint32_t *h_bad = h_len + n;
  uint32_t *d_bad = reinterpret_cast<uint32_t *>(ctx->d_small);
  const BatchDev bd{seq, seq, off, off, len, len};
  ce = cudaMemsetAsync(d_bad, 0, 4, st);
  if (ce == cudaSuccess) ce = launch_validate_pairs(bd, n, 4, d_bad, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_bad, d_bad, 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_len, len, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "reading the lengths");
  ++launches;
  if (*h_bad) {
    set_error("%u codes are 4 or more (RNA codes A=0 C=1 G=2 U=3)", *h_bad);
    return FILTR_ERR_INVALID;
  }
  std::vector<uint64_t> words(n);
  std::vector<uint32_t> h_len_copy(h_len, h_len + n);  // h_stage is reused below
  for (uint32_t p = 0; p < n; ++p) {
    if (h_len[p] > FILTR_FOLD_MAX_LEN) {
      set_error("sequence %u has %u bases; the limit is %u", p, h_len[p], FILTR_FOLD_MAX_LEN);
      return FILTR_ERR_UNSUPPORTED;
    }
    words[p] = (uint64_t)h_len[p] * (h_len[p] + 1) / 2;
  }
  // workspace: order, table offsets, then the tables in waves
  Carve c{ctx->ws, ctx->ws_bytes};
  uint32_t *d_order = c.take<uint32_t>(n);
  uint64_t *d_toff = c.take<uint64_t>(n);
  const size_t tbase = (c.used + 255) / 256 * 256;
  const uint64_t twords = ctx->ws_bytes > tbase ? (ctx->ws_bytes - tbase) / 4 : 0;
  if (!ctx->ensure_host((size_t)n * 12 + 256)) {
    set_error("pinned host allocation failed");
    return FILTR_ERR_NOMEM;
  }
  uint64_t *h_toff = reinterpret_cast<uint64_t *>(ctx->h_stage);
  uint32_t *h_ord = reinterpret_cast<uint32_t *>(h_toff + n);
  std::vector<std::pair<uint32_t, uint32_t>> waves;
  uint64_t used = 0;
  uint32_t begin = 0;
  for (uint32_t p = 0; p < n; ++p) {
    const uint64_t w = (words[p] + 3) / 4 * 4;
    if (w > twords) {
      set_error("sequence %u needs %llu table words; the workspace holds %llu", p,
                (unsigned long long)w, (unsigned long long)twords);
      return FILTR_ERR_NOMEM;
    }
    if (used + w > twords) {
      waves.push_back({begin, p});
      begin = p;
      used = 0;
    }
    h_toff[p] = used;
    h_ord[p] = p;
    used += w;
  }
  waves.push_back({begin, n});
  ce = cudaMemcpyAsync(d_toff, h_toff, (size_t)n * 8, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_order, h_ord, (size_t)n * 4, cudaMemcpyHostToDevice, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "uploading the table layout");
  FoldArgs a{};
  a.seq = seq;
  a.off = off;
  a.len = len;
  a.table_off = d_toff;
  a.table = reinterpret_cast<int32_t *>(ctx->ws + tbase);
  a.out = out;
  a.partner = prm->traceback ? partner : nullptr;
  a.min_loop = prm->min_loop;
  a.use_xdrop = prm->use_xdrop ? 1 : 0;
  a.xdrop = prm->xdrop;
  a.warmup = prm->warmup;
  // thread groups per cell for short sequences only: measured on 1024-2048
  // structured RNAs, grouping took 76 bases 1.14 -> 0.62 ms, 120 bases 2.67 ->
  // 1.54 ms and 300 bases 13.6 -> 11.7 ms, but 500 bases 61 -> 77 ms, whose
  // tables (0.5 MB each) no longer stay in L2 once the group's loads scatter
  uint32_t max_len = 0;
  for (uint32_t p = 0; p < n; ++p) max_len = std::max(max_len, h_len_copy[p]);
  a.max_group = max_len <= 320 ? 32 : 1;
  ctx->span_begin(Ctx::PH_FORWARD, st);
  for (const auto &w : waves) {
    a.order = d_order + w.first;
    k_fold<<<w.second - w.first, FOLD_THREADS, 0, st>>>(a);
    ++launches;
    ce = cudaGetLastError();
    if (ce != cudaSuccess) break;
  }
  ctx->span_end(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "fold kernel");
  ctx->last_waves = (int)waves.size();
  ctx->last_launches = launches;
  ctx->last_cells_estimate = 0;
  ctx->last_cells_packed = 0;
  ctx->last_pairs_packed = 0;
  if (!ctx->done_ev) cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
  if (ctx->done_ev) cudaEventRecord(ctx->done_ev, st);
  return FILTR_OK;
}

}  // namespace filtr

using namespace filtr;

extern "C" filtr_status filtr_fold_batch(filtr_ctx *ctx, const filtr_fold_params *params,
                                         uint32_t n_seqs, const uint8_t *seq, const uint64_t *off,
                                         const uint32_t *len, filtr_fold_result *out,
                                         int32_t *partner, void *stream) {
  if (!ctx) {
    set_error("ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  return fold_impl(reinterpret_cast<Ctx *>(ctx), params, n_seqs, seq, off, len, out, partner,
                   static_cast<cudaStream_t>(stream));
}
