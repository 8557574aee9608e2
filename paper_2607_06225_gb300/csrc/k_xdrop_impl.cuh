// k_xdrop_impl.cuh -- exact antidiagonal sweep for X-drop pruning (Sec. 5.2 / 7.2) and
// Z-drop pruning (Sec. 9.3), optionally intersected with a static band (Sec. 7.1).
// Instantiated by k_xdrop.cu (X-drop), k_zdrop.cu (Z-drop) and k_xdrop_mid.cu
// (X-drop over Table 1's M/I/D recurrence, where gaps open from the diagonal
// state M: one more state array, G, carries M of antidiagonal k-1), which
// compile in parallel.
//
// X-drop decides antidiagonal k from best(k-1), the largest unpruned H of
// antidiagonal k-1 (with FILTR_PRUNE_XDROP_RUNNING the largest of every
// antidiagonal up to k-1), and the diagonal range [lo(k-1), hi(k-1)] of its unpruned
// cells, so antidiagonals are processed strictly one after another: compute all
// cells of k, reduce (max H, min / max diagonal of the unpruned cells), then
// move on.  A group of W warps (one pair) holds a window of WIN = W*32*S slots;
// thread t owns slots [tS, tS+S).  Slot p of antidiagonal k is the cell
// (i, j) = (k - c_k - p, c_k + p): c_k, the window origin, follows the left end
// of the candidate range and advances by delta_k in {0, 1} per antidiagonal, so
// the neighbours of slot p are compile-time offsets:
//   left (i, j-1) on k-1 : slot p - 1 + delta_k
//   up   (i-1, j) on k-1 : slot p + delta_k
//   diag (i-1, j-1) on k-2: slot p - 1 + delta_k + delta_{k-1}
// Values crossing a thread boundary move by __shfl_up/down_sync inside a warp
// and through shared memory between warps; the per-antidiagonal reductions use
// redux.sync (__reduce_max_sync / __reduce_min_sync) plus one barrier for W > 1.
// Residue codes ride along in registers (4 per word) and shift by one slot when
// the window moves; the one code entering a thread's window is loaded directly.
// A pair whose candidate range outgrows the window stops with status TOO_WIDE
// and is rerun by the host with a wider group.
//
// Pruned or out-of-domain cells hold NEG in H, E and F.
#include <climits>

#pragma once

#include "filtr_internal.h"
#include "k_xdrop_layout.h"

namespace filtr {
namespace {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int XS = 8;  // slots per thread

struct Edge {
  int H1, E1, F1, H2;
  int G1;  // M/I/D: the diagonal state M on antidiagonal k-1 (gaps open from it)
};

template <int W>
struct alignas(16) XdShared {
  int red[2][W][4];      // per warp: max H, min slot, max slot of unpruned cells, slot of max H
  Edge first[2][W];      // slot 0 of the warp (lane 0) after each antidiagonal
  Edge last[2][W];       // slot 31*S + S-1 of the warp (lane 31)
  uint32_t pair;         // work item of the group
  unsigned long long rsv;  // traceback rows reserved by the group (checkpointed sweep)
};

__device__ __forceinline__ int code_at(const uint32_t (&w)[2], int s) {
  return (int)((w[s >> 2] >> (8 * (s & 3))) & 0xffu);
}

// shift the 8 codes of a thread up by one slot (slot s <- s-1), new code in slot 0
__device__ __forceinline__ void codes_up(uint32_t (&w)[2], uint32_t in) {
  w[1] = __funnelshift_l(w[0], w[1], 8);
  w[0] = (w[0] << 8) | (in & 0xffu);
}
// shift down by one slot (slot s <- s+1), new code in slot S-1
__device__ __forceinline__ void codes_down(uint32_t (&w)[2], uint32_t in) {
  w[0] = __funnelshift_r(w[0], w[1], 8);
  w[1] = (w[1] >> 8) | ((in & 0xffu) << 24);
}

template <int W, bool LOCAL, bool AFFINE, bool TB, int VAR, int DELTA, int DOFF>
__device__ __forceinline__ void xd_cells(
    int (&H1)[XS], int (&E1)[XS], int (&F1)[XS], int (&H2)[XS], int (&G1)[XS], int (&Hn)[XS],
    int (&En)[XS], int (&Fn)[XS], int (&Gn)[XS], const Edge &pv, const Edge &nx,
    const uint32_t (&qw)[2], const uint32_t (&rw)[2], const int8_t *s_sub, int A, int o, int e,
    int vA, int vB, int thr, int zx, uint32_t &nibs, int &tmax, int &tlo, int &thi,
    int &tbest_slot) {
  constexpr bool ZD = VAR == 1, MIDF = VAR == 2;
  const int oe = o + e;
#pragma unroll
  for (int s = 0; s < XS; ++s) {
    const int ls = s - 1 + DELTA, us = s + DELTA, ds = s + DOFF;
    const int Hl = (ls < 0) ? pv.H1 : H1[ls < 0 ? 0 : ls];
    const int El = (ls < 0) ? pv.E1 : E1[ls < 0 ? 0 : ls];
    const int Hu = (us >= XS) ? nx.H1 : H1[us >= XS ? XS - 1 : us];
    // where a gap opens: H (Gotoh H/E/F) or the diagonal state M (Table 1's M/I/D)
    const int Ol = MIDF ? ((ls < 0) ? pv.G1 : G1[ls < 0 ? 0 : ls]) : Hl;
    const int Ou = MIDF ? ((us >= XS) ? nx.G1 : G1[us >= XS ? XS - 1 : us]) : Hu;
    const int Fu = (us >= XS) ? nx.F1 : F1[us >= XS ? XS - 1 : us];
    const int Hd = (ds < 0) ? pv.H2 : ((ds >= XS) ? nx.H2 : H2[ds < 0 ? 0 : (ds >= XS ? XS - 1 : ds)]);
    const int sc = s_sub[code_at(qw, s) * A + code_at(rw, s)];
    const int D = Hd + sc;
    int E, F, DE, H;
    if (AFFINE) {
      const int Hol = Ol - oe, Eext = El - e, Hou = Ou - oe, Fext = Fu - e;
      E = max(Hol, Eext);
      F = max(Hou, Fext);
      DE = max(D, E);
      H = max(DE, F);
      if (TB) tb_push4(nibs, D - E, DE - F, Hol - Eext, Hou - Fext);
    } else {
      E = Hl - e;
      F = Hu - e;
      DE = max(D, E);
      H = max(DE, F);
      if (TB) tb_push4(nibs, D - E, DE - F, 0, 0);
    }
    if (LOCAL) H = max(H, 0);
    // Z-drop: the threshold falls by the cell's distance from the previous
    // antidiagonal's best diagonal, |d - d_best| = |zx + 2s|
    const int thr_s = ZD ? max(thr - abs(zx + 2 * s), NEG_HALF) : thr;
    const bool alive = (s >= vA) && (s <= vB) && (H >= thr_s);
    if (MIDF) Gn[s] = alive ? D : NEG;
    if (!alive) {
      H = NEG;
      E = NEG;
      F = NEG;
    } else {
      if (H > tmax) {
        tmax = H;
        tbest_slot = s;  // the largest slot wins ties below (smallest i)
      } else if (H == tmax) {
        tbest_slot = s;
      }
      tlo = min(tlo, s);
      thi = max(thi, s);
    }
    Hn[s] = H;
    En[s] = E;
    Fn[s] = F;
  }
}

template <int W, bool LOCAL, bool AFFINE, bool TB, int VAR>
__global__ void __launch_bounds__(W == 1 ? 128 : W * 32) k_xdrop(const FullArgs a, uint32_t *overflow,
                                                              uint32_t *n_overflow) {
  constexpr int WIN = W * 32 * XS;
  constexpr int GROUPS = (W == 1) ? 4 : 1;
  __shared__ XdShared<W> shm[GROUPS];
  __shared__ int8_t s_sub[MAX_ALPHA * MAX_ALPHA];
  const int A = a.sp.alphabet;
  for (int t = threadIdx.x; t < A * A; t += blockDim.x) s_sub[t] = a.sp.subst[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (W == 1) ? 0 : (int)(threadIdx.x >> 5);   // warp inside the group
  const int grp = (W == 1) ? (int)(threadIdx.x >> 5) : 0;
  XdShared<W> &sh = shm[grp];
  const int tid = warp * 32 + lane;  // thread inside the group
  const int o = a.sp.o, e = a.sp.e;
  const int X = a.sp.xdrop;
  const bool no_thresh = (X >= FILTR_XDROP_INF);

  auto gsync = [&]() {
    if (W == 1)
      __syncwarp();
    else
      __syncthreads();
  };

  bool first_item = true;
  for (;;) {
    // ---- next pair --------------------------------------------------------------
    uint32_t t0 = 0;
    if (a.ck) {  // checkpointed sweep: one pair, taken once by group 0
      t0 = (first_item && grp == 0) ? 0u : a.n_order;
      first_item = false;
    } else if (W == 1) {
      if (lane == 0) t0 = atomicAdd(a.counter, 1u);
      t0 = __shfl_sync(FULLMASK, t0, 0);
    } else {
      if (threadIdx.x == 0) sh.pair = atomicAdd(a.counter, 1u);
      __syncthreads();
      t0 = sh.pair;
      __syncthreads();
    }
    if (t0 >= a.n_order) break;
    const uint32_t p = a.order[t0];
    const int M = (int)a.b.q_len[p], N = (int)a.b.r_len[p];
    const uint8_t *q = a.b.q_seq + a.b.q_off[p];
    const uint8_t *r = a.b.r_seq + a.b.r_off[p];
    int64_t blo = -(int64_t)M, bhi = N;
    if (a.sp.use_band) band_limits(M, N, a.sp.band, a.sp.band_literal, &blo, &bhi);
    const int band_lo = (int)max(blo, -(int64_t)M), band_hi = (int)min(bhi, (int64_t)N);

    const XdCkpt *ck = a.ck;
    const int ckmode = ck ? ck->mode : 0;
    const int seg = ck ? ck->k_start / ck->C : 0;
    if (ckmode == 3) {
      // another launch did this segment, the sweep has finished, or the state
      // to resume does not fit this window (every thread reads the same words)
      bool skip = ck->flags[0] != 0 || ck->flags[1 + seg] != 0;
      if (!skip && ck->k_start > 0)
        skip = ck->buf[(int64_t)seg * xd_ckpt_stride() + XCK_USED] > WIN;
      if (skip) break;
    }
    uint32_t *tbp = nullptr;
    int32_t *ckp = nullptr;
    unsigned long long rsv = 0;
    if (TB) {
      if (ckmode == 2) {  // rows indexed by k - k_start - 1
        ckp = ck->seg_ck;
        tbp = ck->seg_tb;
      } else if (ckmode == 3) {  // rows from the pool, indexed by k - k_start - 1
        const unsigned long long need = (unsigned long long)ck->C * (WIN / 8);
        if (W == 1) {
          if (lane == 0) rsv = atomicAdd(ck->pool_next, need);
          rsv = __shfl_sync(FULLMASK, rsv, 0);
        } else {
          if (threadIdx.x == 0) sh.rsv = atomicAdd(ck->pool_next, need);
          __syncthreads();
          rsv = sh.rsv;
          __syncthreads();
        }
        if (rsv + need > ck->pool_words) {  // every thread sees the same rsv
          if (tid == 0) ck->flags[0] = 2;
          break;
        }
        ckp = ck->seg_ck_all + (int64_t)seg * ck->C;
        tbp = ck->pool + rsv;
      } else {
        ckp = reinterpret_cast<int32_t *>(a.tb + a.tbl[p].off);
        tbp = a.tb + a.tbl[p].off + (uint64_t)xd_origin_words(M, N);
      }
    }

    // ---- antidiagonal 0: the cell (0, 0) ---------------------------------------
    constexpr bool ZD = VAR == 1, MIDF = VAR == 2;
    int H1[XS], E1[XS], F1[XS], H2[XS], G1[XS];
#pragma unroll
    for (int s = 0; s < XS; ++s) {
      H1[s] = NEG;
      E1[s] = NEG;
      F1[s] = NEG;
      H2[s] = NEG;
      G1[s] = NEG;
    }
    if (tid == 0) H1[0] = 0;
    if (MIDF && tid == 0) G1[0] = 0;  // every path starts at the origin in the M state
    int c = 0, dprev = 0;  // window origin and its last move
    int best = 0, lo = 0, hi = 0, dbest = 0;  // dbest: diagonal of the best cell (Z-drop)
    // running best cell of this thread: value, i, j (largest H, then smallest i, then j)
    int bv = INT_MIN, bi = INT_MAX, bj = INT_MAX;
    if (tid == 0) {
      bv = 0;
      bi = 0;
      bj = 0;
    }
    uint64_t cells = 0;
    int status = FILTR_ST_OK;
    bool corner = false;
    int cornerH = INT_MIN;  // set by the thread owning (M, N) on antidiagonal M + N
    // residue codes of this thread's slots at the current origin: q[i-1], r[j-1]
    uint32_t qw[2] = {0, 0}, rw[2] = {0, 0};
    if (TB && tid == 0 && ckmode == 0) ckp[0] = 0;
    int k_first = 1, k_last = M + N;
    if (ckmode >= 2) {
      // resume from the checkpoint of antidiagonal k_start
      k_first = ck->k_start + 1;
      k_last = min(ck->k_end, M + N);
      if (ck->k_start > 0) {
        const int32_t *rec = ck->buf + (int64_t)seg * xd_ckpt_stride();
        c = rec[XCK_ORIGIN];
        dprev = rec[XCK_DPREV];
        best = rec[XCK_BEST];
        lo = rec[XCK_LO];
        hi = rec[XCK_HI];
        dbest = rec[XCK_DBEST];
        const int wwin = rec[XCK_WIN];  // slots beyond the writer's window are NEG
        const int32_t *mine = rec + XCK_HDR + tid * (4 * XS);
#pragma unroll
        for (int s = 0; s < XS; ++s) {
          const bool in = tid * XS + s < wwin;
          H1[s] = in ? mine[s] : NEG;
          E1[s] = in ? mine[XS + s] : NEG;
          F1[s] = in ? mine[2 * XS + s] : NEG;
          H2[s] = in ? mine[3 * XS + s] : NEG;
        }
        if (ckmode == 3) {  // the best cell and the cell count so far
          if (tid == 0) {
            bv = rec[XCK_BV];
            bi = rec[XCK_BI];
            bj = rec[XCK_BJ];
          }
          cells = (uint64_t)(uint32_t)rec[XCK_CELLS_LO] | ((uint64_t)(uint32_t)rec[XCK_CELLS_HI] << 32);
        }
      }
    }
    bool ended = false;  // the sweep stopped (empty antidiagonal or k = M + N)
    if (W > 1) {
      const int b0 = (k_first - 1) & 1;
      if (lane == 0) sh.first[b0][warp] = Edge{H1[0], E1[0], F1[0], H2[0], G1[0]};
      if (lane == 31) sh.last[b0][warp] = Edge{H1[XS - 1], E1[XS - 1], F1[XS - 1], H2[XS - 1], G1[XS - 1]};
      __syncthreads();
    }

    int k = k_first;
    for (; k <= k_last; ++k) {
      // ---- candidate range of antidiagonal k, as columns [jA, jB] --------------
      int dl = lo - 1, dh = hi + 1;
      dl = max(dl, band_lo);
      dh = min(dh, band_hi);
      // parity of k; d = 2j - k
      const int jA = max(max(0, k - M), (k + dl + 1) >> 1);  // ceil((k+dl)/2)
      const int jB = min(min(N, k), (k + dh) >> 1);           // floor((k+dh)/2)
      if (jA > jB) {  // empty domain: nothing alive on k
        ended = true;
        break;
      }
      const int cn = min(jA, c + 1);
      const int delta = cn - c;
      if (jB - cn + 1 > WIN) {
        status = FILTR_ST_TOO_WIDE;
        break;
      }
      // residue codes at the new origin: slot p <-> (i, j) = (k - cn - p, cn + p)
      // delta 1: j + 1 for every slot (r shifts down), i same
      // delta 0: i + 1 for every slot (q shifts up), j same
      if (k == k_first) {
        // first fill: load directly
        uint32_t w0 = 0, w1 = 0, v0 = 0, v1 = 0;
#pragma unroll
        for (int s = 0; s < XS; ++s) {
          const int pp = tid * XS + s;
          const int j = cn + pp, i = k - j;
          const uint32_t qc = (i >= 1 && i <= M) ? q[i - 1] : 0u;
          const uint32_t rc = (j >= 1 && j <= N) ? r[j - 1] : 0u;
          if (s < 4) {
            w0 |= qc << (8 * s);
            v0 |= rc << (8 * s);
          } else {
            w1 |= qc << (8 * (s - 4));
            v1 |= rc << (8 * (s - 4));
          }
        }
        qw[0] = w0;
        qw[1] = w1;
        rw[0] = v0;
        rw[1] = v1;
      } else if (delta == 1) {
        const int j = cn + tid * XS + XS - 1;
        codes_down(rw, (j >= 1 && j <= N) ? r[j - 1] : 0u);
      } else {
        const int i = k - cn - tid * XS;
        codes_up(qw, (i >= 1 && i <= M) ? q[i - 1] : 0u);
      }

      // ---- neighbour values across thread boundaries ---------------------------
      Edge pv, nx;
      pv.H1 = __shfl_up_sync(FULLMASK, H1[XS - 1], 1);
      pv.E1 = __shfl_up_sync(FULLMASK, E1[XS - 1], 1);
      pv.F1 = NEG;
      pv.H2 = __shfl_up_sync(FULLMASK, H2[XS - 1], 1);
      nx.H1 = __shfl_down_sync(FULLMASK, H1[0], 1);
      nx.F1 = __shfl_down_sync(FULLMASK, F1[0], 1);
      nx.E1 = NEG;
      nx.H2 = __shfl_down_sync(FULLMASK, H2[0], 1);
      pv.G1 = MIDF ? __shfl_up_sync(FULLMASK, G1[XS - 1], 1) : NEG;
      nx.G1 = MIDF ? __shfl_down_sync(FULLMASK, G1[0], 1) : NEG;
      const int buf = (k - 1) & 1;
      if (lane == 0) {
        if (W > 1 && warp > 0)
          pv = sh.last[buf][warp - 1];
        else
          pv = Edge{NEG, NEG, NEG, NEG, NEG};
      }
      if (lane == 31) {
        if (W > 1 && warp < W - 1)
          nx = sh.first[buf][warp + 1];
        else
          nx = Edge{NEG, NEG, NEG, NEG, NEG};
      }

      // ---- cells of antidiagonal k -------------------------------------------
      const int base_slot = tid * XS;
      const int vA = jA - cn - base_slot, vB = jB - cn - base_slot;
      int thr = NEG_HALF;
      if (!no_thresh) thr = (int)max((long long)best - (long long)X, (long long)NEG_HALF);
      const int zx = ZD ? 2 * (cn + base_slot) - k - dbest : 0;
      int Hn[XS], En[XS], Fn[XS], Gn[XS];
      uint32_t nibs = 0;
      int tmax = INT_MIN, tlo = INT_MAX, thi = INT_MIN, tbs = -1;
      const int doff = delta + dprev - 1;
      // a warp whose slots all lie outside the candidate range only clears its state
      const bool wact = __any_sync(FULLMASK, vB >= 0 && vA < XS);
      if (!wact) {
#pragma unroll
        for (int s = 0; s < XS; ++s) {
          Hn[s] = NEG;
          En[s] = NEG;
          Fn[s] = NEG;
          Gn[s] = NEG;
        }
      } else if (delta == 1) {
        if (doff == 0)
          xd_cells<W, LOCAL, AFFINE, TB, VAR, 1, 0>(H1, E1, F1, H2, G1, Hn, En, Fn, Gn, pv, nx, qw, rw, s_sub, A,
                                              o, e, vA, vB, thr, zx, nibs, tmax, tlo, thi, tbs);
        else
          xd_cells<W, LOCAL, AFFINE, TB, VAR, 1, 1>(H1, E1, F1, H2, G1, Hn, En, Fn, Gn, pv, nx, qw, rw, s_sub, A,
                                              o, e, vA, vB, thr, zx, nibs, tmax, tlo, thi, tbs);
      } else {
        if (doff == 0)
          xd_cells<W, LOCAL, AFFINE, TB, VAR, 0, 0>(H1, E1, F1, H2, G1, Hn, En, Fn, Gn, pv, nx, qw, rw, s_sub, A,
                                              o, e, vA, vB, thr, zx, nibs, tmax, tlo, thi, tbs);
        else
          xd_cells<W, LOCAL, AFFINE, TB, VAR, 0, -1>(H1, E1, F1, H2, G1, Hn, En, Fn, Gn, pv, nx, qw, rw, s_sub,
                                               A, o, e, vA, vB, thr, zx, nibs, tmax, tlo, thi, tbs);
      }
#pragma unroll
      for (int s = 0; s < XS; ++s) {
        H2[s] = H1[s];
        H1[s] = Hn[s];
        E1[s] = En[s];
        F1[s] = Fn[s];
        if (MIDF) G1[s] = Gn[s];
      }
      if (TB) {
        // only the 32-byte sectors (8 threads) of the row that hold a slot of
        // the candidate range: the walk reads no other
        const int64_t row = (ckmode >= 2) ? (int64_t)(k - ck->k_start - 1) : (int64_t)k;
        const unsigned act = __ballot_sync(FULLMASK, vB >= 0 && vA < XS);
        if ((act >> (lane & 24)) & 0xffu) tbp[row * (WIN / 8) + tid] = nibs;
        if (tid == 0) ckp[row] = cn;
      }
      // this thread's best cell on k (largest slot among equal maxima = smallest i)
      if (tbs >= 0) {
        const int jj = cn + base_slot + tbs, ii = k - jj;
        if (tmax > bv || (tmax == bv && (ii < bi || (ii == bi && jj < bj)))) {
          bv = tmax;
          bi = ii;
          bj = jj;
        }
      }
      // cells with i >= 1 and j >= 1 in the candidate range
      {
        const int a0 = max(jA, 1), b0 = min(jB, k - 1);
        if (b0 >= a0) cells += (uint64_t)(b0 - a0 + 1);
      }
      // the corner (M, N) is the single cell of antidiagonal M + N
      if (k == M + N) {
        const int pc = N - cn;  // its slot
        if (pc >= base_slot && pc < base_slot + XS) {
#pragma unroll
          for (int s = 0; s < XS; ++s)
            if (base_slot + s == pc) cornerH = H1[s];
        }
      }

      // ---- reductions over the group ---------------------------------------------
      const int wmax = __reduce_max_sync(FULLMASK, tmax);
      const int wlo = __reduce_min_sync(FULLMASK, tlo == INT_MAX ? INT_MAX : base_slot + tlo);
      const int whi = __reduce_max_sync(FULLMASK, thi == INT_MIN ? INT_MIN : base_slot + thi);
      // Z-drop: the largest slot holding the maximum (the best cell with the
      // smallest i, whose diagonal the next antidiagonal measures from)
      int wbs = -1;
      if (ZD) wbs = __reduce_max_sync(FULLMASK, (tbs >= 0 && tmax == wmax) ? base_slot + tbs : -1);
      int gmax = wmax, glo = wlo, ghi = whi, gbs = wbs;
      if (W > 1) {
        const int nb = k & 1;
        if (lane == 0) {
          sh.red[nb][warp][0] = wmax;
          sh.red[nb][warp][1] = wlo;
          sh.red[nb][warp][2] = whi;
          if (ZD) sh.red[nb][warp][3] = wbs;
          sh.first[nb][warp] = Edge{H1[0], E1[0], F1[0], H2[0], G1[0]};
        }
        if (lane == 31) sh.last[nb][warp] = Edge{H1[XS - 1], E1[XS - 1], F1[XS - 1], H2[XS - 1], G1[XS - 1]};
        __syncthreads();
#pragma unroll
        for (int w = 0; w < W; ++w) {
          gmax = max(gmax, sh.red[nb][w][0]);
          glo = min(glo, sh.red[nb][w][1]);
          ghi = max(ghi, sh.red[nb][w][2]);
        }
        if (ZD) {
          gbs = -1;
#pragma unroll
          for (int w = 0; w < W; ++w)
            if (sh.red[nb][w][0] == gmax) gbs = max(gbs, sh.red[nb][w][3]);
        }
      }
      c = cn;
      dprev = delta;
      if (glo == INT_MAX) {  // nothing alive on k: the sweep ends here
        if (k == M + N) corner = false;
        ended = true;
        break;
      }
      if (!a.sp.xrun || gmax > best) {  // running best: the first maximum keeps its diagonal
        best = gmax;
        if (ZD) dbest = 2 * (cn + gbs) - k;
      }
      lo = 2 * (cn + glo) - k;
      hi = 2 * (cn + ghi) - k;
      if (k == M + N) corner = true;
    }
    if (k > k_last && k_last == M + N) ended = true;
    // a window too narrow for this segment leaves it to the next, wider launch
    if (ckmode == 3 && status == FILTR_ST_TOO_WIDE && W < XD_MAX_WARPS) break;

    // ---- result -------------------------------------------------------------------
    // group-wide best cell (largest H, then smallest i, then smallest j)
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const int ov = __shfl_down_sync(FULLMASK, bv, off);
      const int oi = __shfl_down_sync(FULLMASK, bi, off);
      const int oj = __shfl_down_sync(FULLMASK, bj, off);
      if (ov > bv || (ov == bv && (oi < bi || (oi == bi && oj < bj)))) {
        bv = ov;
        bi = oi;
        bj = oj;
      }
    }
    if (W > 1) {
      __syncthreads();
      if (lane == 0) {
        sh.red[0][warp][0] = bv;
        sh.red[0][warp][1] = bi;
        sh.red[0][warp][2] = bj;
      }
      __syncthreads();
      bv = sh.red[0][0][0];
      bi = sh.red[0][0][1];
      bj = sh.red[0][0][2];
      for (int w = 1; w < W; ++w) {
        const int ov = sh.red[0][w][0], oi = sh.red[0][w][1], oj = sh.red[0][w][2];
        if (ov > bv || (ov == bv && (oi < bi || (oi == bi && oj < bj)))) {
          bv = ov;
          bi = oi;
          bj = oj;
        }
      }
    }
    // the corner value lives in one thread; broadcast it
    if (!LOCAL) {
      int ch = __reduce_max_sync(FULLMASK, cornerH);
      if (W > 1) {
        __syncthreads();
        if (lane == 0) sh.red[1][warp][0] = ch;
        __syncthreads();
        ch = INT_MIN;
        for (int w = 0; w < W; ++w) ch = max(ch, sh.red[1][w][0]);
      }
      cornerH = ch;
    }
    if (ckmode == 3 && !ended && status == FILTR_ST_OK) {
      // segment done, sweep not finished: store the window state after k_end
      int32_t *rec = ck->buf + (int64_t)(ck->k_end / ck->C) * xd_ckpt_stride();
      int used = 0;  // one past the last slot holding a value other than NEG
#pragma unroll
      for (int s = 0; s < XS; ++s)
        if (H1[s] != NEG || E1[s] != NEG || F1[s] != NEG || H2[s] != NEG) used = tid * XS + s + 1;
      used = __reduce_max_sync(FULLMASK, used);
      if (W > 1) {
        __syncthreads();
        if (lane == 0) sh.red[0][warp][0] = used;
        __syncthreads();
        for (int w = 0; w < W; ++w) used = max(used, sh.red[0][w][0]);
      }
      int32_t *mine = rec + XCK_HDR + tid * (4 * XS);
#pragma unroll
      for (int s = 0; s < XS; ++s) {
        mine[s] = H1[s];
        mine[XS + s] = E1[s];
        mine[2 * XS + s] = F1[s];
        mine[3 * XS + s] = H2[s];
      }
      if (tid == 0) {
        rec[XCK_ORIGIN] = c;
        rec[XCK_DPREV] = dprev;
        rec[XCK_BEST] = best;
        rec[XCK_LO] = lo;
        rec[XCK_HI] = hi;
        rec[XCK_DBEST] = dbest;
        rec[XCK_USED] = used;
        rec[XCK_WIN] = WIN;
        rec[XCK_BV] = bv;
        rec[XCK_BI] = bi;
        rec[XCK_BJ] = bj;
        rec[XCK_CELLS_LO] = (int32_t)(uint32_t)cells;
        rec[XCK_CELLS_HI] = (int32_t)(uint32_t)(cells >> 32);
        if (TB) {
          ck->seg_off[seg] = rsv;
          ck->seg_w[seg] = W;
        }
        ck->flags[1 + seg] = W;
      }
      gsync();
      continue;
    }
    if (tid == 0 && ckmode != 2) {
      if (ckmode == 3) {  // the sweep ends in this segment (or outgrew the widest window)
        if (TB && status != FILTR_ST_TOO_WIDE) {
          ck->seg_off[seg] = rsv;
          ck->seg_w[seg] = W;
        }
        ck->flags[0] = 1;
        if (status != FILTR_ST_TOO_WIDE) ck->flags[1 + seg] = W;
      }
      int score = 0, ei = 0, ej = 0;
      if (status == FILTR_ST_TOO_WIDE) {
        const uint32_t slot = atomicAdd(n_overflow, 1u);
        overflow[slot] = p;
      } else if (LOCAL) {
        if (bv > 0) {
          score = bv;
          ei = bi;
          ej = bj;
        } else {
          status = FILTR_ST_EMPTY;
        }
      } else if (corner) {
        score = cornerH;
        ei = M;
        ej = N;
      } else {
        status = FILTR_ST_DROPPED;
        score = bv;
        ei = bi;
        ej = bj;
      }
      filtr_result res;
      res.score = score;
      res.q_end = ei;
      res.r_end = ej;
      res.q_begin = (LOCAL && status == FILTR_ST_OK) ? -1 : 0;
      res.r_begin = res.q_begin;
      res.status = status;
      res.cigar_len = 0;
      res.reserved = 0;
      res.cigar_off = 0;
      res.cells = cells;
      a.out[p] = res;
      FwdOut f;
      f.score = score;
      f.end_i = ei;
      f.end_j = ej;
      f.status = status;
      a.fwd[p] = f;
    }
    gsync();
  }
}

template <int W, bool LOCAL, bool AFFINE, bool TB, int VAR>
cudaError_t launch_w(const FullArgs &a, int grid, uint32_t *ovf, uint32_t *novf, cudaStream_t s) {
  k_xdrop<W, LOCAL, AFFINE, TB, VAR><<<grid, W == 1 ? 128 : W * 32, 0, s>>>(a, ovf, novf);
  return cudaGetLastError();
}

template <int W, int VAR>
cudaError_t dispatch_w(const FullArgs &a, int grid, uint32_t *ovf, uint32_t *novf, cudaStream_t s) {
  const bool L = a.sp.mode == FILTR_LOCAL, AF = a.sp.affine != 0, T = a.sp.traceback != 0;
  if constexpr (VAR == 2) {  // M/I/D: affine gaps only
    if (!AF) return cudaErrorInvalidValue;
    if (L)
      return T ? launch_w<W, true, true, true, VAR>(a, grid, ovf, novf, s)
               : launch_w<W, true, true, false, VAR>(a, grid, ovf, novf, s);
    return T ? launch_w<W, false, true, true, VAR>(a, grid, ovf, novf, s)
             : launch_w<W, false, true, false, VAR>(a, grid, ovf, novf, s);
  }
  if (L) {
    if (AF)
      return T ? launch_w<W, true, true, true, VAR>(a, grid, ovf, novf, s)
               : launch_w<W, true, true, false, VAR>(a, grid, ovf, novf, s);
    return T ? launch_w<W, true, false, true, VAR>(a, grid, ovf, novf, s)
             : launch_w<W, true, false, false, VAR>(a, grid, ovf, novf, s);
  }
  if (AF)
    return T ? launch_w<W, false, true, true, VAR>(a, grid, ovf, novf, s)
             : launch_w<W, false, true, false, VAR>(a, grid, ovf, novf, s);
  return T ? launch_w<W, false, false, true, VAR>(a, grid, ovf, novf, s)
           : launch_w<W, false, false, false, VAR>(a, grid, ovf, novf, s);
}

template <int W, bool LOCAL, bool AFFINE, bool TB, int VAR>
int occ_xd() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_xdrop<W, LOCAL, AFFINE, TB, VAR>,
                                                W == 1 ? 128 : W * 32, 0);
  return nb;
}

template <int W, int VAR>
int occ_w(const ScoreParams &sp) {
  const bool L = sp.mode == FILTR_LOCAL, AF = sp.affine != 0, T = sp.traceback != 0;
  if constexpr (VAR == 2) {
    if (!AF) return 0;
    if (L) return T ? occ_xd<W, true, true, true, VAR>() : occ_xd<W, true, true, false, VAR>();
    return T ? occ_xd<W, false, true, true, VAR>() : occ_xd<W, false, true, false, VAR>();
  }
  if (L) {
    if (AF) return T ? occ_xd<W, true, true, true, VAR>() : occ_xd<W, true, true, false, VAR>();
    return T ? occ_xd<W, true, false, true, VAR>() : occ_xd<W, true, false, false, VAR>();
  }
  if (AF) return T ? occ_xd<W, false, true, true, VAR>() : occ_xd<W, false, true, false, VAR>();
  return T ? occ_xd<W, false, false, true, VAR>() : occ_xd<W, false, false, false, VAR>();
}

template <int VAR>
cudaError_t launch_any_w(const FullArgs &a, int W, int grid, uint32_t *ovf, uint32_t *novf,
                         cudaStream_t s) {
  switch (W) {
    case 1: return dispatch_w<1, VAR>(a, grid, ovf, novf, s);
    case 2: return dispatch_w<2, VAR>(a, grid, ovf, novf, s);
    case 4: return dispatch_w<4, VAR>(a, grid, ovf, novf, s);
    case 8: return dispatch_w<8, VAR>(a, grid, ovf, novf, s);
    case 16: return dispatch_w<16, VAR>(a, grid, ovf, novf, s);
    case 32: return dispatch_w<32, VAR>(a, grid, ovf, novf, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int VAR>
int occ_any_w(int W, const ScoreParams &sp) {
  switch (W) {
    case 1: return occ_w<1, VAR>(sp);
    case 2: return occ_w<2, VAR>(sp);
    case 4: return occ_w<4, VAR>(sp);
    case 8: return occ_w<8, VAR>(sp);
    case 16: return occ_w<16, VAR>(sp);
    case 32: return occ_w<32, VAR>(sp);
    default: return 0;
  }
}

}  // namespace
}  // namespace filtr
