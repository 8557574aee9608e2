// search.cu -- edit distance by the search traversal (Sec. 6.3): the kernel and
// the filtr_search_batch entry point.
//
// One warp per pair, persistent over a work queue.  Wavefront s holds, for each
// diagonal d = j - i of its domain, the furthest row s edits reach:
//   F[s][d] = extend(max(F[s-1][d] + 1, F[s-1][d+1] + 1, F[s-1][d-1]))
// (mismatch, a step down from diagonal d+1, a step right from diagonal d-1),
// each term only when its predecessor was reached and the move stays inside the
// matrix; extend() follows matches.  Lane l of the warp takes the diagonals
// lo + l, lo + l + 32, ...; each lane loads its diagonal of the previous
// wavefront once and takes the neighbours d - 1 and d + 1 by warp shuffles
// (a chunk's edge lanes from the neighbouring chunk or one extra load).  Both
// sequences are staged in shared memory, so a match run compares four residues
// per step (two aligned words each side and a funnel shift).  The domain grows by one diagonal on each side per score, clipped to
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

#include "../../include/filtr_testing.h"
#include "filtr_ctx.h"

namespace filtr {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int UNREACHED = -1;
constexpr uint32_t OP_I = 1, OP_D = 2, OP_EQ = 7, OP_X = 8;
constexpr int SEARCH_CHUNKS = 4;  // chunks of 32 diagonals a warp has in flight per iteration

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
  uint32_t ring_c;            // score pass: entries of each shared-memory ring (power of two)
  int band;                   // < 0: none
  int adapt_min, adapt_max;   // adapt_min == 0: exact
};

// Four residues starting at byte i of a staged sequence.
__device__ __forceinline__ uint32_t load4(const uint32_t *w, int i) {
  const uint32_t a = w[i >> 2], b = w[(i >> 2) + 1];
  return __funnelshift_r(a, b, (i & 3) * 8);
}

// A sequence staged in shared memory: residue i at byte ph + i of w.
struct Staged {
  const uint32_t *w;
  int ph;
};

// Sixteen 2-bit residues starting at residue i of a packed sequence.
__device__ __forceinline__ uint32_t load16(const uint32_t *w, int i) {
  const uint32_t a = w[i >> 4], b = w[(i >> 4) + 1];
  return __funnelshift_r(a, b, (i & 15) * 2);
}

// The free transitions: row reached from row i on diagonal d by matches, four
// byte residues (P2: sixteen 2-bit residues) per comparison.
template <bool P2>
__device__ __forceinline__ int extend(const Staged &q, const Staged &r, int i, int d, int M,
                                      int N) {
  constexpr int K = P2 ? 16 : 4, B = P2 ? 2 : 8;
  int rem = min(M - i, N - i - d);  // residues left on the diagonal
  int qi = q.ph + i, ri = r.ph + i + d;
  while (rem > 0) {
    uint32_t x = P2 ? (load16(q.w, qi) ^ load16(r.w, ri)) : (load4(q.w, qi) ^ load4(r.w, ri));
    if (rem < K) x |= 0xffffffffu << (B * rem);  // residues past an end never match
    if (x) return qi - q.ph + ((__ffs(x) - 1) / B);
    qi += K;
    ri += K;
    rem -= K;
  }
  return qi - q.ph + rem;  // rem <= 0: back to the end of the diagonal
}

// Copy the 16-byte blocks that hold g[0, len) into dst (16-byte aligned) with
// 16-byte loads; returns the byte of dst that holds g[0].  The blocks lie
// within g's own 16-byte-aligned span, so no load crosses a page.
// P2 (codes 0..3): each 16-byte block becomes one word of 2-bit codes, so
// residue i again sits at position ph + i, counted in 2-bit units.
__device__ __forceinline__ uint32_t pack_bytes2(uint32_t x) {  // four codes < 4 -> 8 bits
  return (x & 3u) | ((x >> 6) & 0xcu) | ((x >> 12) & 0x30u) | ((x >> 18) & 0xc0u);
}
template <bool P2>
__device__ __forceinline__ int stage_seq(const uint8_t *g, int len, uint32_t *dst, int lane) {
  const uintptr_t ga = reinterpret_cast<uintptr_t>(g);
  const int ph = (int)(ga & 15u);
  const uint4 *src = reinterpret_cast<const uint4 *>(ga - (uintptr_t)ph);
  const int nblk = len > 0 ? (ph + len + 15) >> 4 : 0;
  if (P2) {
    for (int k = lane; k < nblk; k += 32) {
      const uint4 v = __ldg(src + k);
      dst[k] = pack_bytes2(v.x) | (pack_bytes2(v.y) << 8) | (pack_bytes2(v.z) << 16) |
               (pack_bytes2(v.w) << 24);
    }
  } else {
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int k = lane; k < nblk; k += 32) d4[k] = __ldg(src + k);
  }
  return ph;
}

// Where a wavefront's values live: level s in b0 (s even) or b1 (s odd), the
// value of diagonal d at index (d + off) & mask -- a power-of-two ring in shared
// memory (off 0, mask C - 1: two's complement wraps negative d) or a buffer of
// M + N + 1 entries in global memory (off M, mask all ones).
struct Wf {
  int *b0, *b1;
  int off;
  uint32_t mask;
};
__device__ __forceinline__ int at(int d, int off, uint32_t mask) {
  return (int)((uint32_t)(d + off) & mask);
}
__device__ __forceinline__ int *level_buf(const Wf &w, int s) { return (s & 1) ? w.b1 : w.b0; }

// Largest term of F[s][d] from the previous wavefront pv (alive diagonals
// [palo, pahi]); UNREACHED when none exists.  *which: 0 mismatch, 1 insertion,
// 2 deletion (the first in that order on ties).
__device__ __forceinline__ int terms(const int *pv, int off, uint32_t mask, int palo, int pahi,
                                     int d, int M, int N, int *which) {
  int best = UNREACHED, w = -1;
  if (d >= palo && d <= pahi) {
    const int v = pv[at(d, off, mask)];
    if (v >= 0 && v + 1 <= M && v + 1 + d <= N) {
      best = v + 1;
      w = 0;
    }
  }
  if (d + 1 >= palo && d + 1 <= pahi) {
    const int v = pv[at(d + 1, off, mask)];
    if (v >= 0 && v + 1 <= M && v + 1 > best) {
      best = v + 1;
      w = 1;
    }
  }
  if (d - 1 >= palo && d - 1 <= pahi) {
    const int v = pv[at(d - 1, off, mask)];
    if (v >= 0 && v + d <= N && v > best) {
      best = v;
      w = 2;
    }
  }
  *which = w;
  return best;
}

// WFA-Adapt: the diagonals of [lo, hi] that survive -- reached, and remaining
// distance max(M - i, N - j) within amax of the wavefront's smallest; the
// bounds move inwards to the outermost survivors.
__device__ __forceinline__ void adapt_bounds(const int *cv, int off, uint32_t mask, int lo, int hi,
                                             int M, int N, int amax, int lane, int *alo,
                                             int *ahi) {
  int rmin = INT_MAX;
  for (int d0 = lo; d0 <= hi; d0 += 32) {
    const int d = d0 + lane;
    if (d <= hi) {
      const int f = cv[at(d, off, mask)];
      if (f >= 0) rmin = min(rmin, max(M - f, N - f - d));
    }
  }
  rmin = __reduce_min_sync(FULL, rmin);
  int qlo = INT_MAX, qhi = INT_MIN;
  for (int d0 = lo; d0 <= hi; d0 += 32) {
    const int d = d0 + lane;
    if (d <= hi) {
      const int f = cv[at(d, off, mask)];
      if (f >= 0 && max(M - f, N - f - d) - rmin <= amax) {
        qlo = min(qlo, d);
        qhi = max(qhi, d);
      }
    }
  }
  *alo = __reduce_min_sync(FULL, qlo);
  *ahi = __reduce_max_sync(FULL, qhi);
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

// One pair's shape, shared by both passes.
struct PairView {
  int M, N, dlo, dhi, target;
  Staged q, r;
};

// Stage the pair's sequences in shared memory and set up its domain limits.
template <bool P2>
__device__ __forceinline__ PairView stage_pair(const SearchArgs &a, uint32_t p, uint32_t *sq,
                                               uint32_t *sr, int lane) {
  PairView v;
  v.M = (int)a.b.q_len[p];
  v.N = (int)a.b.r_len[p];
  v.q = Staged{sq, stage_seq<P2>(a.b.q_seq + a.b.q_off[p], v.M, sq, lane)};
  v.r = Staged{sr, stage_seq<P2>(a.b.r_seq + a.b.r_off[p], v.N, sr, lane)};
  __syncwarp();
  v.dlo = -v.M;
  v.dhi = v.N;
  if (a.band >= 0) {
    v.dlo = max(v.dlo, min(0, v.N - v.M) - a.band);
    v.dhi = min(v.dhi, max(0, v.N - v.M) + a.band);
  }
  v.target = v.N - v.M;
  return v;
}

// Progress of one pair's search.
struct Lev {
  int lo, hi, s;
  uint64_t cells;
  int state;  // 0 running, 1 reached (M, N), 2 gave up (not expected)
};

// Score levels from L.s on, until (M, N) is reached or -- in a shared-memory
// ring of C entries -- the next wavefront would not fit (state stays 0).
template <bool SMEM, int CH, bool P2>
__device__ __forceinline__ void levels(Lev &L, const Wf &w, int C, const PairView &v, int amin,
                                       int amax, int lane) {
  const int M = v.M, N = v.N;
  for (;;) {
    const int *cv = level_buf(w, L.s);
    bool done = false;
    if (lane == 0 && v.target >= L.lo && v.target <= L.hi)
      done = cv[at(v.target, w.off, w.mask)] >= M;
    done = __shfl_sync(FULL, done, 0);
    if (done) {
      L.state = 1;
      return;
    }
    int alo = L.lo, ahi = L.hi;
    if (amin > 0 && L.hi - L.lo + 1 >= amin)
      adapt_bounds(cv, w.off, w.mask, L.lo, L.hi, M, N, amax, lane, &alo, &ahi);
    if (L.s >= M + N + 1 || alo > ahi) {  // the leading diagonal always survives
      L.state = 2;
      return;
    }
    const int nlo = max(alo - 1, v.dlo), nhi = min(ahi + 1, v.dhi);
    if (SMEM && nhi - nlo + 1 > C) return;
    int *nv = level_buf(w, L.s + 1);
    // CH chunks of 32 diagonals per iteration: one load per diagonal of the
    // previous wavefront (alive diagonals only); the neighbours d - 1 and d + 1
    // by two rotating shuffles, in which lane 31 (lane 0) hands lane 0 (lane 31)
    // the last (first) diagonal of the chunk before (after) instead of its own
    const uint32_t mk = SMEM ? w.mask : 0xffffffffu;
    for (int d0 = nlo; d0 <= nhi; d0 += 32 * CH) {
      int vc[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int d = d0 + 32 * u + lane;
        vc[u] = (d >= alo && d <= ahi) ? cv[at(d, w.off, mk)] : UNREACHED;
      }
      const int dl = d0 - 1, dr = d0 + 32 * CH;  // outer edges: lane 31 / lane 0 load them
      const int el = (lane == 31 && dl >= alo && dl <= ahi) ? cv[at(dl, w.off, mk)] : UNREACHED;
      const int er = (lane == 0 && dr >= alo && dr <= ahi) ? cv[at(dr, w.off, mk)] : UNREACHED;
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int d = d0 + 32 * u + lane;
        const int to_right = lane == 31 ? (u > 0 ? vc[u > 0 ? u - 1 : 0] : el) : vc[u];
        const int to_left = lane == 0 ? (u + 1 < CH ? vc[u + 1 < CH ? u + 1 : 0] : er) : vc[u];
        const int vl = __shfl_sync(FULL, to_right, (lane + 31) & 31);  // F[s][d - 1]
        const int vr = __shfl_sync(FULL, to_left, (lane + 1) & 31);    // F[s][d + 1]
        int row = UNREACHED;
        if (vc[u] >= 0 && vc[u] + 1 <= M && vc[u] + 1 + d <= N) row = vc[u] + 1;  // mismatch
        if (vr >= 0 && vr + 1 <= M && vr + 1 > row) row = vr + 1;                // insertion
        if (vl >= 0 && vl + d <= N && vl > row) row = vl;                        // deletion
        if (d <= nhi) nv[at(d, w.off, mk)] = row >= 0 ? extend<P2>(v.q, v.r, row, d, M, N) : UNREACHED;
      }
    }
    __syncwarp();
    L.cells += (uint64_t)(nhi - nlo + 1);
    L.lo = nlo;
    L.hi = nhi;
    ++L.s;
  }
}

// Score pass: distance and wavefront cells of every pair, and the words its
// traceback pass would store.  Per warp in shared memory: the two sequences,
// then two rings of ring_c entries; a pair whose wavefront outgrows them moves
// to the warp's buffers in global memory.
template <bool P2>
__global__ void __launch_bounds__(128) k_search_score(const SearchArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t *sq = smem + (size_t)wib * (a.q_words + a.r_words + 2 * a.ring_c);
  uint32_t *sr = sq + a.q_words;
  int *ra = reinterpret_cast<int *>(sr + a.r_words), *rb = ra + a.ring_c;
  const uint64_t slot = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  int *g = a.ring + slot * 2 * a.ring_half;
  const Wf ws{ra, rb, 0, a.ring_c - 1u};

  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= a.n) return;
    const uint32_t p = a.order ? a.order[t] : t;
    const PairView v = stage_pair<P2>(a, p, sq, sr, lane);
    // score 0: the origin and its run of matches
    if (lane == 0) ra[at(0, ws.off, ws.mask)] = extend<P2>(v.q, v.r, 0, 0, v.M, v.N);
    __syncwarp();
    Lev L{0, 0, 0, 1ull, 0};
    levels<true, SEARCH_CHUNKS, P2>(L, ws, (int)a.ring_c, v, a.adapt_min, a.adapt_max, lane);
    if (L.state == 0) {  // level L.s to global memory, then on from there
      const Wf wg{g, g + a.ring_half, v.M, 0xffffffffu};
      const int *src = level_buf(ws, L.s);
      int *dst = level_buf(wg, L.s);
      for (int d = L.lo + lane; d <= L.hi; d += 32)
        dst[at(d, wg.off, wg.mask)] = src[at(d, ws.off, ws.mask)];
      __syncwarp();
      levels<false, SEARCH_CHUNKS, P2>(L, wg, 0, v, a.adapt_min, a.adapt_max, lane);
    }
    if (lane == 0) {
      const bool ok = L.state == 1;
      filtr_result r;
      r.score = ok ? -L.s : 0;
      r.q_begin = 0;
      r.q_end = v.M;
      r.r_begin = 0;
      r.r_end = v.N;
      r.status = ok ? FILTR_ST_OK : FILTR_ST_TOO_WIDE;
      r.cigar_len = 0;
      r.reserved = 0;
      r.cigar_off = 0;
      r.cells = L.cells;
      a.out[p] = r;
      if (a.need) a.need[p] = ok ? 4ull * (uint64_t)(L.s + 1) + L.cells : 0ull;
    }
    __syncwarp();
  }
}

// Traceback pass: the same levels again, every wavefront kept in the pair's
// store (per score: lo, hi and the alive bounds, then the values), then lane 0
// walks back from (M, N).
template <bool P2>
__global__ void __launch_bounds__(128) k_search_tb(const SearchArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t *sq = smem + (size_t)wib * (a.q_words + a.r_words);
  uint32_t *sr = sq + a.q_words;

  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= a.n) return;
    const uint32_t p = a.order ? a.order[t] : t;
    if (a.out[p].status != FILTR_ST_OK) {  // the score pass gave up on it (not expected)
      if (lane == 0) a.out[p].cigar_len = 0;
      continue;
    }
    const PairView v = stage_pair<P2>(a, p, sq, sr, lane);
    const int M = v.M, N = v.N;
    const int S = -a.out[p].score;
    int *meta = a.arena + a.arena_off[p];  // per score: lo, hi, alo, ahi
    int *waves = meta + 4 * (S + 1);
    int lo = 0, hi = 0;
    int *cv = waves;
    uint64_t woff = 0;
    if (lane == 0) cv[0] = extend<P2>(v.q, v.r, 0, 0, M, N);
    __syncwarp();
    int s = 0;
    bool ok = true;
    for (;;) {
      bool done = false;
      if (v.target >= lo && v.target <= hi && lane == 0) done = cv[v.target - lo] >= M;
      done = __shfl_sync(FULL, done, 0);
      int alo = lo, ahi = hi;
      if (!done && a.adapt_min > 0 && hi - lo + 1 >= a.adapt_min)
        adapt_bounds(cv, -lo, 0xffffffffu, lo, hi, M, N, a.adapt_max, lane, &alo, &ahi);
      if (lane == 0) {
        meta[4 * s + 0] = lo;
        meta[4 * s + 1] = hi;
        meta[4 * s + 2] = alo;
        meta[4 * s + 3] = ahi;
      }
      if (done) break;
      if (s >= S || alo > ahi) {  // not expected: the score pass reached (M, N) at S
        ok = false;
        break;
      }
      const int *pv = cv;
      const int pbase = lo;
      const int nlo = max(alo - 1, v.dlo), nhi = min(ahi + 1, v.dhi);
      woff += (uint64_t)(hi - lo + 1);
      cv = waves + woff;
      for (int d0 = nlo; d0 <= nhi; d0 += 32) {
        const int d = d0 + lane;
        if (d <= nhi) {
          int which;
          const int row = terms(pv, -pbase, 0xffffffffu, alo, ahi, d, M, N, &which);
          cv[d - nlo] = row >= 0 ? extend<P2>(v.q, v.r, row, d, M, N) : UNREACHED;
        }
      }
      __syncwarp();
      lo = nlo;
      hi = nhi;
      ++s;
    }
    if (lane == 0) {
      // walk back from (M, N): per score, the matches after the edit, then the edit
      RevEmitter em{a.stage + a.stage_off[p]};
      if (ok) {
        int d = v.target, i = M;
        for (int u = s; u > 0; --u) {
          const int plo = meta[4 * (u - 1)], phi = meta[4 * (u - 1) + 1];
          const int palo = meta[4 * (u - 1) + 2], pahi = meta[4 * (u - 1) + 3];
          woff -= (uint64_t)(phi - plo + 1);
          int which;
          const int row = terms(waves + woff, -plo, 0xffffffffu, palo, pahi, d, M, N, &which);
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

// Block shape of a kernel with `wbytes` of shared memory per warp: the warps per
// block (4, 2 or 1) that keep the most warps resident per SM.
struct LaunchCfg {
  int wpb = 1, per_sm = 0;
  size_t smem = 0;
};
template <class K>
cudaError_t pick_cfg(K kern, size_t wbytes, LaunchCfg *cfg) {
  LaunchCfg best;
  for (int wpb : {4, 2, 1}) {
    const size_t smem = wbytes * wpb;
    if (smem > 227 * 1024) continue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, smem);
    if (e != cudaSuccess) return e;
    if (per_sm * wpb > best.per_sm * best.wpb) best = LaunchCfg{wpb, per_sm, smem};
  }
  if (best.per_sm < 1) return cudaErrorInvalidConfiguration;
  *cfg = best;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best.smem);
}

// One persistent launch of at most max_warps warps.
template <class K>
cudaError_t launch_cfg(K kern, const LaunchCfg &cfg, const SearchArgs &a, int sms,
                       uint64_t max_warps, cudaStream_t st) {
  const uint64_t want = ((uint64_t)a.n + cfg.wpb - 1) / cfg.wpb;
  const uint64_t grid =
      std::min<uint64_t>(std::min<uint64_t>(want, (uint64_t)sms * cfg.per_sm), max_warps / cfg.wpb);
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned)grid, 32 * cfg.wpb, cfg.smem, st>>>(a);
  return cudaGetLastError();
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
  if (prm->alphabet != 0 && prm->alphabet != 4) {
    set_error("search alphabet must be 0 (any byte codes) or 4 (DNA codes 0..3)");
    return FILTR_ERR_INVALID;
  }
  const bool p2 = prm->alphabet == 4;
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
  ce = cudaSuccess;
  uint32_t *h_ql = reinterpret_cast<uint32_t *>(ctx->h_stage), *h_rl = h_ql + n;
  uint32_t *h_bad = h_rl + n;
  uint32_t *d_bad = reinterpret_cast<uint32_t *>(ctx->d_small);
  *h_bad = 0;
  if (p2) {  // DNA codes are packed two bits each: every code must be below 4
    ce = cudaMemsetAsync(d_bad, 0, 4, st);
    if (ce == cudaSuccess) ce = launch_validate_pairs(b, n, 4, d_bad, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_bad, d_bad, 4, cudaMemcpyDeviceToHost, st);
    ++launches;
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_ql, b.q_len, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_rl, b.r_len, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "reading the lengths");
  if (*h_bad) {
    set_error("%u residue codes are 4 or more (search alphabet 4)", *h_bad);
    return FILTR_ERR_INVALID;
  }
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
  // staging: the 16-byte blocks holding a sequence (up to 15 bytes before its
  // first residue) and the word after its last, in whole 16-byte blocks
  // (P2: one word per block, and the word after the last residue's)
  a.q_words = p2 ? (max_m + 48) / 64 * 4 + 4 : (max_m + 48) / 16 * 4;
  a.r_words = p2 ? (max_n + 48) / 64 * 4 + 4 : (max_n + 48) / 16 * 4;
  a.ring_half = max_m + max_n + 1;
  // shared-memory rings: small, so they cost little occupancy; a pair whose
  // wavefront grows wider continues in global memory
  const uint32_t ring_cap = ctx->search_ring > 0 ? (uint32_t)ctx->search_ring : 32u;
  a.ring_c = 32;
  while (a.ring_c < a.ring_half && a.ring_c < ring_cap) a.ring_c <<= 1;
  LaunchCfg cfg_score, cfg_tb;
  auto k_score = p2 ? k_search_score<true> : k_search_score<false>;
  auto k_tb = p2 ? k_search_tb<true> : k_search_tb<false>;
  ce = pick_cfg(k_score, (size_t)(a.q_words + a.r_words + 2 * a.ring_c) * 4, &cfg_score);
  if (ce == cudaSuccess && tb) ce = pick_cfg(k_tb, (size_t)(a.q_words + a.r_words) * 4, &cfg_tb);
  if (ce != cudaSuccess) return cuda_fail(ce, "search kernel occupancy");

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
  // global buffers for wavefronts that outgrow the rings: one per resident warp,
  // no more warps than pairs, no more than the workspace holds
  const uint64_t slot_bytes = 2ull * a.ring_half * sizeof(int);
  const int wpb = cfg_score.wpb;
  uint64_t n_slots = std::min<uint64_t>((uint64_t)ctx->sms * cfg_score.per_sm * wpb,
                                        ((uint64_t)n + wpb - 1) / wpb * wpb);
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
  ce = launch_cfg(k_score, cfg_score, a, ctx->sms, n_slots, st);
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
      ce = launch_cfg(k_tb, cfg_tb, a, ctx->sms, UINT64_MAX, st);
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
  ctx->last_cells_packed = 0;
  ctx->last_pairs_packed = 0;
  if (!ctx->done_ev) cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
  if (ctx->done_ev) cudaEventRecord(ctx->done_ev, st);
  return FILTR_OK;
}

}  // namespace filtr

using namespace filtr;

extern "C" filtr_status filtr_test_set_search_ring(filtr_ctx *ctx, int32_t entries) {
  if (!ctx || (entries != 0 && (entries < 32 || entries > 4096 || (entries & (entries - 1))))) {
    set_error("filtr_test_set_search_ring: bad arguments");
    return FILTR_ERR_INVALID;
  }
  reinterpret_cast<Ctx *>(ctx)->search_ring = entries;
  return FILTR_OK;
}

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
