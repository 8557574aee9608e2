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
// of R/8 words per lane; the high half of a lane's rows runs one step behind.
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
  const int wps = g.R / 8;
  const uint32_t w =
      __ldg(tb + s * g.strip_words + (t * wps + h * (P / 8) + (k >> 3)) * 32 + l);
  const int c = k & 7;
  return (((w >> c) & 1u) << 3) | (((w >> (8 + c)) & 1u) << 2) | (((w >> (16 + c)) & 1u) << 1) |
         ((w >> (24 + c)) & 1u);
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

__global__ void k_walk(const WalkArgs a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_order) return;
  const uint32_t p = a.order[t];
  const FwdOut f = a.fwd[p];
  const TbLayout L = a.tbl[p];
  if (f.status != FILTR_ST_OK && f.status != FILTR_ST_DROPPED) {
    a.out[p].cigar_len = 0;
    return;
  }
  const int M = (int)a.b.q_len[p], N = (int)a.b.r_len[p];
  const uint8_t *q = a.b.q_seq + a.b.q_off[p];
  const uint8_t *r = a.b.r_seq + a.b.r_off[p];
  const bool local = a.sp.mode == FILTR_LOCAL;
  const int A = a.sp.alphabet, e = a.sp.e, oe = a.sp.o + a.sp.e;
  const uint32_t *tb = a.tb + L.off;

  FullGeom g;
  XdGeom xg;
  PackGeom pg{L.R, (int64_t)pack_strip_tb_words(1, N, L.R)};
  if (L.family == FAM_FULL && L.valid) {
    g.R = L.R;
    g.HS = 32 * L.R;
    g.M = M;
    g.N = N;
    g.band = a.sp.use_band != 0;
    band_limits(M, N, a.sp.band, a.sp.band_literal, &g.lo, &g.hi);
    if (!g.band) {
      g.lo = -(int64_t)M - 1;
      g.hi = (int64_t)N + 1;
    }
    // start at the strip holding the last row, base = sum of earlier strips
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
        state = 0;
      }
      --j;
    } else {
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
        state = 0;
      }
      --i;
    }
  }
  em.flush();
  filtr_result *res = a.out + p;
  res->q_begin = i;
  res->r_begin = j;
  res->cigar_len = em.n;
}

// Resumable walk over one recomputed segment (antidiagonals (k_start, k_end])
// of a checkpointed X-drop traceback; one thread.  Stops when the walk leaves
// the segment (the next, earlier segment continues from the saved state) or
// when the alignment's start is reached.
__global__ void k_walk_segment(const WalkArgs a, const uint32_t *seg_tb, const int32_t *seg_ck,
                               int k_start, int wpk, WalkState *ws) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  WalkState w = *ws;
  if (w.done) return;
  const uint32_t p = a.order[0];
  const uint8_t *q = a.b.q_seq + a.b.q_off[p];
  const uint8_t *r = a.b.r_seq + a.b.r_off[p];
  const bool local = a.sp.mode == FILTR_LOCAL;
  const int A = a.sp.alphabet, e = a.sp.e, oe = a.sp.o + a.sp.e;
  Emitter em{a.stage + a.stage_off[p], w.n, w.cur, w.run};
  int i = w.i, j = w.j, v = w.v, state = w.state;
  bool done = false;
  auto bits = [&](int ii, int jj) -> uint32_t {
    const int64_t row = (int64_t)ii + jj - k_start - 1;
    const int pp = jj - seg_ck[row];
    return tb_nibble(seg_tb[row * wpk + (pp >> 3)], pp);
  };
  for (;;) {
    if (state == 0) {
      if ((i == 0 && j == 0) || (local && v == 0)) {
        done = true;
        break;
      }
      if (i == 0) {
        em.put(OP_D, (uint32_t)j);
        j = 0;
        done = true;
        break;
      }
      if (j == 0) {
        em.put(OP_I, (uint32_t)i);
        i = 0;
        done = true;
        break;
      }
    }
    if (i + j <= k_start) break;  // the cell belongs to an earlier segment
    if (state == 0) {
      const uint32_t nib = bits(i, j);
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
      const uint32_t nib = bits(i, j);
      em.put(OP_D, 1);
      if (nib & TB_EEXT) {
        v += e;
      } else {
        v += oe;
        state = 0;
      }
      --j;
    } else {
      if (i == 0) {
        state = 0;
        continue;
      }
      const uint32_t nib = bits(i, j);
      em.put(OP_I, 1);
      if (nib & TB_FEXT) {
        v += e;
      } else {
        v += oe;
        state = 0;
      }
      --i;
    }
  }
  if (done) {
    em.flush();
    filtr_result *res = a.out + p;
    res->q_begin = i;
    res->r_begin = j;
    res->cigar_len = em.n;
  }
  w.i = i;
  w.j = j;
  w.v = v;
  w.state = state;
  w.done = done ? 1 : 0;
  w.n = em.n;
  w.cur = em.cur;
  w.run = em.run;
  *ws = w;
}

// Exclusive scan of cigar_len (pair order) into offs; *total = sum.  One CTA.
__global__ void k_scan(const filtr_result *out, uint32_t n, uint64_t *offs, uint64_t *total) {
  __shared__ uint64_t part[1024];
  __shared__ uint64_t carry;
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
  k_walk<<<(a.n_order + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_walk_segment(const WalkArgs &a, const uint32_t *seg_tb, const int32_t *seg_ck,
                                int k_start, int wpk, WalkState *st, cudaStream_t s) {
  k_walk_segment<<<1, 32, 0, s>>>(a, seg_tb, seg_ck, k_start, wpk, st);
  return cudaGetLastError();
}

cudaError_t launch_scan_offsets(const filtr_result *out, uint32_t n, uint64_t *offs,
                                uint64_t *total, cudaStream_t s) {
  k_scan<<<1, 1024, 0, s>>>(out, n, offs, total);
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
