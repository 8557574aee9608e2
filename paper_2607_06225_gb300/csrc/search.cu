// search.cu -- edit distance by the search traversal (Sec. 6.3): the kernel and
// the filtr_search_batch entry point.
//
// One warp per pair, persistent over a work queue.  Wavefront s holds, for each
// diagonal d = j - i of its domain, the furthest row s edits reach:
//   F[s][d] = extend(max(F[s-1][d] + 1, F[s-1][d+1] + 1, F[s-1][d-1]))
// (mismatch, a step down from diagonal d+1, a step right from diagonal d-1),
// each term only when its predecessor was reached and the move stays inside the
// matrix; extend() follows matches.  Lane l of the warp takes the diagonals
// lo + l, lo + l + 32, ...; the three terms are three coalesced loads of the
// previous wavefront.  Both sequences are staged in shared memory, so a match
// run compares four residues per step (two aligned words each side and a funnel
// shift).  The domain grows by one diagonal on each side per score, clipped to
// the matrix and the band; WFA-Adapt (Sec. 7.2, 9.3) moves its bounds inwards
// past unreached diagonals and those whose remaining distance max(M - i, N - j)
// exceeds the wavefront's smallest by more than max_dist, from the first
// wavefront that spans min_len diagonals.
//
// Score pass: the previous and current wavefronts live in a per-warp ring in
// global memory (index d + M, so no copy when the domain moves).  Traceback
// pass: every wavefront is kept (per score its bounds, then its values), its
// size known from the score pass, and one lane walks back from (M, N), taking
// at each score the first of mismatch, insertion, deletion that gives the
// level's value; the ops go to the CIGAR staging area reversed, as the other
// walks leave them.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "filtr_ctx.h"

namespace filtr {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int UNREACHED = -1;
constexpr uint32_t OP_I = 1, OP_D = 2, OP_EQ = 7, OP_X = 8;

struct SearchArgs {
  BatchDev b;
  uint32_t n;                 // pairs of this launch: order[0, n), or 0..n-1
  const uint32_t *order;
  uint32_t *counter;          // work-queue cursor (zeroed before the launch)
  filtr_result *out;
  uint64_t *need;             // score pass: words the traceback pass stores per pair
  int *ring;                  // score pass: per warp slot, two wavefronts of ring_half ints
  uint32_t ring_half;         // >= M + N + 1 of every pair
  int *arena;                 // traceback pass: wavefront store
  const uint64_t *arena_off;  // per pair id
  uint32_t *stage;            // traceback pass: reversed CIGAR ops, per pair id
  const uint64_t *stage_off;
  uint32_t q_words, r_words;  // shared-memory staging per warp (32-bit words)
  int band;                   // < 0: none
  int adapt_min, adapt_max;   // adapt_min == 0: exact
};

// Four residues starting at byte i of a staged sequence.
__device__ __forceinline__ uint32_t load4(const uint32_t *w, int i) {
  const uint32_t a = w[i >> 2], b = w[(i >> 2) + 1];
  return __funnelshift_r(a, b, (i & 3) * 8);
}

// The free transitions: row reached from row i on diagonal d by matches.
__device__ __forceinline__ int extend(const uint32_t *sq, const uint32_t *sr, int i, int d,
                                      int M, int N) {
  for (;;) {
    const int rem = min(M - i, N - i - d);
    if (rem <= 0) return i;
    uint32_t x = load4(sq, i) ^ load4(sr, i + d);
    if (rem < 4) x |= 0xffffffffu << (8 * rem);  // residues past an end never match
    if (x) return i + ((__ffs(x) - 1) >> 3);
    i += 4;
  }
}

// Largest term of F[s][d] from the previous wavefront pv (values at pv[d - pbase],
// alive diagonals [palo, pahi]); UNREACHED when none exists.  *which: 0 mismatch,
// 1 insertion, 2 deletion (the first in that order on ties).
__device__ __forceinline__ int terms(const int *pv, int pbase, int palo, int pahi, int d, int M,
                                     int N, int *which) {
  int best = UNREACHED, w = -1;
  if (d >= palo && d <= pahi) {
    const int v = pv[d - pbase];
    if (v >= 0 && v + 1 <= M && v + 1 + d <= N) {
      best = v + 1;
      w = 0;
    }
  }
  if (d + 1 >= palo && d + 1 <= pahi) {
    const int v = pv[d + 1 - pbase];
    if (v >= 0 && v + 1 <= M && v + 1 > best) {
      best = v + 1;
      w = 1;
    }
  }
  if (d - 1 >= palo && d - 1 <= pahi) {
    const int v = pv[d - 1 - pbase];
    if (v >= 0 && v + d <= N && v > best) {
      best = v;
      w = 2;
    }
  }
  *which = w;
  return best;
}

// Run-length ops, written last op first.
struct RevEmitter {
  uint32_t *dst;
  uint32_t n = 0, op = 0, len = 0;
  __device__ void put(uint32_t o, uint32_t l) {
    if (l == 0) return;
    if (o == op) {
      len += l;
      return;
    }
    if (len) dst[n++] = (len << 4) | op;
    op = o;
    len = l;
  }
  __device__ void flush() {
    if (len) dst[n++] = (len << 4) | op;
    len = 0;
  }
};

template <bool TB>
__global__ void __launch_bounds__(128) k_search(const SearchArgs a) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t *sq = smem + (size_t)wib * (a.q_words + a.r_words);
  uint32_t *sr = sq + a.q_words;
  const uint64_t slot = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  int *ring = TB ? nullptr : a.ring + slot * 2 * a.ring_half;

  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= a.n) return;
    const uint32_t p = a.order ? a.order[t] : t;
    if (TB && a.out[p].status != FILTR_ST_OK) {  // the score pass gave up on it (not expected)
      if (lane == 0) a.out[p].cigar_len = 0;
      continue;
    }
    const int M = (int)a.b.q_len[p], N = (int)a.b.r_len[p];
    const uint8_t *gq = a.b.q_seq + a.b.q_off[p], *gr = a.b.r_seq + a.b.r_off[p];
    uint8_t *sq8 = reinterpret_cast<uint8_t *>(sq), *sr8 = reinterpret_cast<uint8_t *>(sr);
    for (int x = lane; x < M; x += 32) sq8[x] = gq[x];
    for (int x = lane; x < N; x += 32) sr8[x] = gr[x];
    __syncwarp();

    int dlo = -M, dhi = N;
    if (a.band >= 0) {
      dlo = max(dlo, min(0, N - M) - a.band);
      dhi = min(dhi, max(0, N - M) + a.band);
    }
    const int target = N - M;
    int S = 0;
    if (TB) S = -a.out[p].score;
    int *meta = TB ? a.arena + a.arena_off[p] : nullptr;  // per score: lo, hi, alo, ahi
    int *waves = TB ? meta + 4 * (S + 1) : nullptr;

    // score 0: the origin and its run of matches
    int lo = 0, hi = 0;
    int *cv = TB ? waves : ring;
    int cbase = TB ? 0 : -M;
    uint64_t woff = 0, cells = 1;
    {
      const int f = lane == 0 ? extend(sq, sr, 0, 0, M, N) : 0;
      if (lane == 0) cv[0 - cbase] = f;
    }
    __syncwarp();
    int s = 0;
    bool ok = true;
    for (;;) {
      // reached (M, N)?
      bool done = false;
      if (target >= lo && target <= hi && lane == 0) done = cv[target - cbase] >= M;
      done = __shfl_sync(FULL, done, 0);
      int alo = lo, ahi = hi;
      if (!done && a.adapt_min > 0 && hi - lo + 1 >= a.adapt_min) {
        int rmin = INT_MAX;
        for (int d0 = lo; d0 <= hi; d0 += 32) {
          const int d = d0 + lane;
          if (d <= hi) {
            const int f = cv[d - cbase];
            if (f >= 0) rmin = min(rmin, max(M - f, N - f - d));
          }
        }
        rmin = __reduce_min_sync(FULL, rmin);
        int qlo = INT_MAX, qhi = INT_MIN;
        for (int d0 = lo; d0 <= hi; d0 += 32) {
          const int d = d0 + lane;
          if (d <= hi) {
            const int f = cv[d - cbase];
            if (f >= 0 && max(M - f, N - f - d) - rmin <= a.adapt_max) {
              qlo = min(qlo, d);
              qhi = max(qhi, d);
            }
          }
        }
        alo = __reduce_min_sync(FULL, qlo);
        ahi = __reduce_max_sync(FULL, qhi);
      }
      if (TB && lane == 0) {
        meta[4 * s + 0] = lo;
        meta[4 * s + 1] = hi;
        meta[4 * s + 2] = alo;
        meta[4 * s + 3] = ahi;
      }
      if (done) break;
      if (s >= M + N + 1 || alo > ahi || (TB && s >= S)) {
        // not expected: the leading diagonal always survives and the search reaches (M, N)
        ok = false;
        break;
      }
      // next wavefront
      const int *pv = cv;
      const int pbase = cbase;
      const int nlo = max(alo - 1, dlo), nhi = min(ahi + 1, dhi);
      if (TB) {
        woff += (uint64_t)(hi - lo + 1);
        cv = waves + woff;
        cbase = nlo;
      } else {
        cv = ring + ((s + 1) & 1) * a.ring_half;
      }
      for (int d0 = nlo; d0 <= nhi; d0 += 32) {
        const int d = d0 + lane;
        if (d <= nhi) {
          int which;
          const int row = terms(pv, pbase, alo, ahi, d, M, N, &which);
          cv[d - cbase] = row >= 0 ? extend(sq, sr, row, d, M, N) : UNREACHED;
        }
      }
      __syncwarp();
      cells += (uint64_t)(nhi - nlo + 1);
      lo = nlo;
      hi = nhi;
      ++s;
    }

    if (!TB) {
      if (lane == 0) {
        filtr_result r;
        r.score = ok ? -s : 0;
        r.q_begin = 0;
        r.q_end = M;
        r.r_begin = 0;
        r.r_end = N;
        r.status = ok ? FILTR_ST_OK : FILTR_ST_TOO_WIDE;
        r.cigar_len = 0;
        r.reserved = 0;
        r.cigar_off = 0;
        r.cells = cells;
        a.out[p] = r;
        if (a.need) a.need[p] = ok ? 4ull * (uint64_t)(s + 1) + cells : 0ull;
      }
    } else if (lane == 0) {
      // walk back from (M, N): per score, the matches after the edit, then the edit
      RevEmitter em{a.stage + a.stage_off[p]};
      if (ok) {
        int d = target, i = M;
        for (int u = s; u > 0; --u) {
          const int plo = meta[4 * (u - 1)], phi = meta[4 * (u - 1) + 1];
          const int palo = meta[4 * (u - 1) + 2], pahi = meta[4 * (u - 1) + 3];
          woff -= (uint64_t)(phi - plo + 1);
          int which;
          const int row = terms(waves + woff, plo, palo, pahi, d, M, N, &which);
          em.put(OP_EQ, (uint32_t)(i - row));
          if (which == 0) {
            em.put(OP_X, 1);
            i = row - 1;
          } else if (which == 1) {
            em.put(OP_I, 1);
            i = row - 1;
            d = d + 1;
          } else {
            em.put(OP_D, 1);
            i = row;
            d = d - 1;
          }
        }
        em.put(OP_EQ, (uint32_t)i);
      }
      em.flush();
      a.out[p].cigar_len = em.n;
    }
    __syncwarp();
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

// Warps per block for a per-warp shared-memory staging of `bytes`.
int search_warps_per_block(size_t bytes) {
  if (bytes * 4 <= 64 * 1024) return 4;
  if (bytes * 2 <= 96 * 1024) return 2;
  return 1;
}

// One persistent launch: at most max_warps warps (the score pass's ring slots).
template <bool TB>
cudaError_t launch_search(const SearchArgs &a, int sms, uint64_t max_warps, cudaStream_t st) {
  const size_t wbytes = (size_t)(a.q_words + a.r_words) * 4;
  const int wpb = search_warps_per_block(wbytes);
  const size_t smem = wbytes * wpb;
  cudaError_t e = cudaFuncSetAttribute(k_search<TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search<TB>, 32 * wpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = ((uint64_t)a.n + wpb - 1) / wpb;
  const int grid = (int)std::min<uint64_t>(std::min<uint64_t>(want, (uint64_t)sms * per_sm),
                                           max_warps / wpb);
  if (grid == 0) return cudaSuccess;
  k_search<TB><<<grid, 32 * wpb, smem, st>>>(a);
  return cudaGetLastError();
}

// Resident warps of the score pass, rounded to whole blocks (sizes its ring).
int search_slots(size_t wbytes, int sms) {
  const int wpb = search_warps_per_block(wbytes);
  const size_t smem = wbytes * wpb;
  if (cudaFuncSetAttribute(k_search<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return -1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search<false>, 32 * wpb, smem) !=
      cudaSuccess)
    return -1;
  return std::max(per_sm, 1) * sms * wpb;
}

}  // namespace

static filtr_status search_impl(Ctx *ctx, const filtr_search_params *prm, uint32_t n,
                                const BatchDev &b, filtr_result *out, uint32_t *cigar,
                                uint64_t cap, cudaStream_t st) {
  if (!prm) {
    set_error("params is NULL");
    return FILTR_ERR_INVALID;
  }
  if (prm->adapt_min_len < 0 || prm->adapt_max_dist < 0) {
    set_error("WFA-Adapt thresholds must be >= 0");
    return FILTR_ERR_INVALID;
  }
  if (n == 0) return FILTR_OK;
  if (!b.q_seq || !b.r_seq || !b.q_off || !b.r_off || !b.q_len || !b.r_len || !out) {
    set_error("a batch pointer is NULL");
    return FILTR_ERR_INVALID;
  }
  const bool tb = prm->traceback != 0;
  if (tb && !cigar && cap > 0) {
    set_error("cigar is NULL but cigar_cap > 0");
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

  // lengths to the host
  if (!ctx->ensure_host((size_t)n * 8 + 256)) {
    set_error("pinned host allocation failed");
    return FILTR_ERR_NOMEM;
  }
  uint32_t *h_ql = reinterpret_cast<uint32_t *>(ctx->h_stage), *h_rl = h_ql + n;
  ce = cudaMemcpyAsync(h_ql, b.q_len, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_rl, b.r_len, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "reading the lengths");
  uint32_t max_m = 0, max_n = 0;
  uint64_t stage_words = 0;
  for (uint32_t p = 0; p < n; ++p) {
    if ((uint64_t)h_ql[p] + h_rl[p] > FILTR_SEARCH_MAX_LEN) {
      set_error("pair %u: M + N = %llu exceeds %u", p,
                (unsigned long long)h_ql[p] + h_rl[p], FILTR_SEARCH_MAX_LEN);
      return FILTR_ERR_UNSUPPORTED;
    }
    max_m = std::max(max_m, h_ql[p]);
    max_n = std::max(max_n, h_rl[p]);
    stage_words += (uint64_t)h_ql[p] + h_rl[p] + 1;
  }
  std::vector<uint32_t> ql(h_ql, h_ql + n), rl(h_rl, h_rl + n);  // h_stage is reused below

  SearchArgs a{};
  a.b = b;
  a.out = out;
  a.band = prm->band;
  a.adapt_min = prm->adapt_min_len;
  a.adapt_max = prm->adapt_max_dist;
  a.q_words = (max_m + 8) / 4 + 1;
  a.r_words = (max_n + 8) / 4 + 1;
  a.ring_half = max_m + max_n + 1;
  const size_t wbytes = (size_t)(a.q_words + a.r_words) * 4;
  const int slots = search_slots(wbytes, ctx->sms);
  if (slots < 0) return cuda_fail(cudaGetLastError(), "search kernel occupancy");

  Carve c{ctx->ws, ctx->ws_bytes};
  uint32_t *d_counter = c.take<uint32_t>(64);
  uint64_t *d_need = tb ? c.take<uint64_t>(n) : nullptr;
  uint64_t *d_arena_off = tb ? c.take<uint64_t>(n) : nullptr;
  uint64_t *d_stage_off = tb ? c.take<uint64_t>(n) : nullptr;
  uint32_t *d_order = tb ? c.take<uint32_t>(n) : nullptr;
  uint64_t *d_offs = tb ? c.take<uint64_t>(n) : nullptr;
  uint64_t *d_total = tb ? c.take<uint64_t>(4) : nullptr;
  uint32_t *d_stage = tb ? c.take<uint32_t>(stage_words) : nullptr;
  const size_t ring_mark = c.used;
  // ring slots: no more warps than pairs, and no more than the workspace holds
  const uint64_t slot_bytes = 2ull * a.ring_half * sizeof(int);
  const int wpb = search_warps_per_block(wbytes);
  uint64_t n_slots = std::min<uint64_t>((uint64_t)slots, ((uint64_t)n + wpb - 1) / wpb * wpb);
  const size_t ring_base = (c.used + 255) / 256 * 256;
  const uint64_t fit = ctx->ws_bytes > ring_base ? (ctx->ws_bytes - ring_base) / slot_bytes : 0;
  n_slots = std::min<uint64_t>(n_slots, fit / wpb * wpb);
  int *d_ring = c.take<int>((size_t)n_slots * 2 * a.ring_half);
  if (n_slots == 0 || c.used > ctx->ws_bytes) {
    set_error("workspace of %zu bytes is too small for the search (%zu bytes)", ctx->ws_bytes,
              ring_base + (size_t)slot_bytes * wpb);
    return FILTR_ERR_NOMEM;
  }
  ce = cudaMemsetAsync(d_counter, 0, 64 * sizeof(uint32_t), st);
  if (ce != cudaSuccess) return cuda_fail(ce, "clearing the queue counters");

  // score pass
  a.n = n;
  a.counter = d_counter;
  a.need = d_need;
  a.ring = d_ring;
  ctx->span_begin(Ctx::PH_FORWARD, st);
  ce = launch_search<false>(a, ctx->sms, n_slots, st);
  ctx->span_end(st);
  ++launches;
  if (ce != cudaSuccess) return cuda_fail(ce, "search score pass");

  if (tb) {
    // wavefront storage per pair, cut into waves that fit the workspace
    uint64_t *h_need = reinterpret_cast<uint64_t *>(ctx->h_stage);
    ce = cudaMemcpyAsync(h_need, d_need, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "reading the wavefront sizes");
    std::vector<uint64_t> need(h_need, h_need + n);
    c.used = ring_mark;  // the ring is free again: the arena takes the rest
    const size_t arena_base = (c.used + 255) / 256 * 256;
    const uint64_t arena_words =
        ctx->ws_bytes > arena_base ? (ctx->ws_bytes - arena_base) / sizeof(int) : 0;
    int *d_arena = reinterpret_cast<int *>(ctx->ws + arena_base);
    if (!ctx->ensure_host((size_t)n * 8 * 2 + (size_t)n * 4 + 256)) {
      set_error("pinned host allocation failed");
      return FILTR_ERR_NOMEM;
    }
    uint64_t *h_aoff = reinterpret_cast<uint64_t *>(ctx->h_stage);
    uint64_t *h_soff = h_aoff + n;
    uint32_t *h_ord = reinterpret_cast<uint32_t *>(h_soff + n);
    std::vector<std::pair<uint32_t, uint32_t>> wave_ranges;
    uint64_t used = 0, soff = 0;
    uint32_t begin = 0;
    for (uint32_t p = 0; p < n; ++p) {
      const uint64_t w = (need[p] + 3) / 4 * 4;  // keep each pair's store 16-byte aligned
      if (w > arena_words) {
        set_error("pair %u keeps %llu wavefront words; the workspace holds %llu", p,
                  (unsigned long long)w, (unsigned long long)arena_words);
        return FILTR_ERR_NOMEM;
      }
      if (used + w > arena_words) {
        wave_ranges.push_back({begin, p});
        begin = p;
        used = 0;
      }
      h_aoff[p] = used;
      used += w;
      h_ord[p] = p;
      h_soff[p] = soff;
      soff += (uint64_t)ql[p] + rl[p] + 1;
    }
    wave_ranges.push_back({begin, n});
    if (wave_ranges.size() > 60) {
      set_error("the traceback would take %zu waves", wave_ranges.size());
      return FILTR_ERR_NOMEM;
    }
    ce = cudaMemcpyAsync(d_arena_off, h_aoff, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_stage_off, h_soff, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_order, h_ord, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "uploading the traceback layout");
    a.need = nullptr;
    a.ring = nullptr;
    a.arena = d_arena;
    a.arena_off = d_arena_off;
    a.stage = d_stage;
    a.stage_off = d_stage_off;
    ctx->span_begin(Ctx::PH_WALK, st);
    for (size_t w = 0; w < wave_ranges.size(); ++w) {
      a.order = d_order + wave_ranges[w].first;
      a.n = wave_ranges[w].second - wave_ranges[w].first;
      a.counter = d_counter + 1 + w;
      ce = launch_search<true>(a, ctx->sms, UINT64_MAX, st);
      ++launches;
      if (ce != cudaSuccess) break;
    }
    ctx->span_end(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "search traceback pass");
    ctx->last_waves = (int)wave_ranges.size();

    // CIGARs in pair order
    WalkArgs wa{};
    wa.stage = d_stage;
    wa.stage_off = d_stage_off;
    ctx->span_begin(Ctx::PH_PLACE, st);
    ce = launch_scan_offsets(out, n, d_offs, d_total, st);
    if (ce == cudaSuccess) ce = launch_compact(wa, n, d_offs, cigar, cap, out, st);
    ctx->span_end(st);
    launches += 2;
    if (ce != cudaSuccess) return cuda_fail(ce, "CIGAR placement");
    uint64_t *h_total = reinterpret_cast<uint64_t *>(ctx->h_stage);
    ce = cudaMemcpyAsync(h_total, d_total, 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "reading the CIGAR total");
    if (*h_total > cap) {
      set_error("CIGARs need %llu ops, cigar_cap is %llu", (unsigned long long)*h_total,
                (unsigned long long)cap);
      ctx->last_launches = launches;
      return FILTR_ERR_CIGAR_CAP;
    }
  } else {
    ctx->last_waves = 1;
  }
  ctx->last_launches = launches;
  ctx->last_cells_estimate = 0;
  ctx->last_pairs_packed = 0;
  if (!ctx->done_ev) cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
  if (ctx->done_ev) cudaEventRecord(ctx->done_ev, st);
  return FILTR_OK;
}

}  // namespace filtr

using namespace filtr;

extern "C" filtr_status filtr_search_batch(filtr_ctx *ctx, const filtr_search_params *params,
                                           uint32_t n_pairs, const uint8_t *q_seq,
                                           const uint64_t *q_off, const uint32_t *q_len,
                                           const uint8_t *r_seq, const uint64_t *r_off,
                                           const uint32_t *r_len, filtr_result *out,
                                           uint32_t *cigar, uint64_t cigar_cap, void *stream) {
  if (!ctx) {
    set_error("ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  BatchDev b{q_seq, r_seq, q_off, r_off, q_len, r_len};
  return search_impl(c, params, n_pairs, b, out, cigar, cigar_cap,
                     static_cast<cudaStream_t>(stream));  // NULL: the default stream
}
