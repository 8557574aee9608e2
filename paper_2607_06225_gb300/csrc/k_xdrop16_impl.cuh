// k_xdrop16_impl.cuh -- the antidiagonal X-drop / Z-drop sweep (Sec. 5.2 / 7.2,
// Sec. 9.3) with two cells in each 32-bit register (int16x2), for affine
// Gotoh H/E/F alignments.  Instantiated by k_xdrop16.cu (X-drop) and
// k_zdrop16.cu (Z-drop).  The int32 sweep (k_xdrop_impl.cuh) computes the same
// cells; this one trades its per-cell bookkeeping for packed DPX arithmetic.
//
// Values.  Under X-drop every value that can still reach an unpruned cell lies
// within about X of the previous antidiagonal's best, so a group holds values
// relative to a base score b: a real value v is the signed 16-bit v - b + C0.
// When the best drifts more than X16_REBASE from C0 the group moves b (every
// state register shifted by one DPX add with a floor at zero).  Packed 0 is
// minus infinity: every add that can fall below zero goes through a DPX
// add-max with a zero floor (__viaddmax_s16x2_relu), so a pruned or missing
// neighbour stays at 0, and values formed from it (at most the largest
// substitution score) stay far below every threshold.  The host sends a pair
// here only when its threshold leaves room (X <= X16_MAX_DROP); a pair whose
// best nevertheless leaves the range, or whose lowest threshold falls to the
// floor, stops with status X16_OVERFLOW and is rerun by the int32 sweep.
//
// Layout.  Thread t owns slots 8t .. 8t+7 of the window, as in the int32 sweep
// (slot p of antidiagonal k is the cell (k - c_k - p, c_k + p)); register r of
// each state array holds slot r in its low half and slot r + 4 in its high
// half, so the neighbour at slot offset -1 / +1 is register r -/+ 1 for both
// halves, and only registers 0 and 3 take a byte permute with the edge value
// of the next / previous thread.  Traceback nibbles are the int32 sweep's
// (slot s in bits 4(7-s)..4(7-s)+3 of the thread's word), so every walk reads
// both kernels' output alike.  A one-warp group can also hold 16 slots per
// thread (G = 2, a 512-slot window): registers 4g .. 4g+3 then hold slots
// 8g .. 8g+7 as above, each group of four registers behaving like one 8-slot
// thread (its own traceback word, its neighbour views across the group edge
// taken from the other group), so the window's rows and checkpoint records are
// those of two warps of 8-slot threads.
//
// Schedule.  Pruning antidiagonal k needs best(k-1) and the live range
// [lo(k-1), hi(k-1)]; the raw update of k needs only the pruned values of k-1
// and k-2 and the window origin.  The origin follows a lower bound of the left
// end of k's candidate range that lo(k-2) already gives (the range moves left
// by at most one diagonal per antidiagonal), so the reductions of k-1 are in
// flight while the raw cells of k are computed, and are consumed only to mask
// them.  The window may trail the left end by a slot; a pair whose range
// outgrows it is rerun wider (status TOO_WIDE), as in the int32 sweep.
#include <algorithm>
#include <climits>

#pragma once

#include "filtr_internal.h"
#include "k_xdrop_layout.h"

namespace filtr {
namespace {

constexpr unsigned X16_FULL = 0xffffffffu;
constexpr int X16_C0 = 16384;

struct alignas(16) Edge16 {
  uint32_t H1, E1, F1, H2;
};

template <int W>
struct alignas(16) X16Shared {
  int red[2][W][4];  // per warp: max H (packed), lowest live slot, highest live slot, slot of the max
  Edge16 first[2][W];
  Edge16 last[2][W];
  uint32_t pair;
  unsigned long long rsv;
};

// 0xffff in each half whose bit 15 (low) / bit 31 (high) is set, else 0
__device__ __forceinline__ uint32_t x16_halfmask(uint32_t x) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, 0xbb99;" : "=r"(r) : "r"(x));
  return r;
}
// per half [a > b] in bit 15 / 31, for halves in [0, 0x7fff]
__device__ __forceinline__ uint32_t x16_gt(uint32_t a, uint32_t b) { return a + 0x7fff7fffu - b; }
// per half [a >= b] in bit 15 / 31, for halves in [0, 0x7fff]
__device__ __forceinline__ uint32_t x16_ge(uint32_t a, uint32_t b) { return a + 0x80008000u - b; }
// register view of the slots one below: slot r - 1 (low) and r + 3 (high); for
// register 0 the low half is the previous thread's slot 7 (high half of pv)
__device__ __forceinline__ uint32_t x16_down0(uint32_t x3, uint32_t pv) { return __byte_perm(x3, pv, 0x1076); }
// register view of the slots one above for register 3: slot 4 (high half of
// x0) and the next thread's slot 0 (low half of nx)
__device__ __forceinline__ uint32_t x16_up3(uint32_t x0, uint32_t nx) { return __byte_perm(x0, nx, 0x5432); }
__device__ __forceinline__ uint32_t x16_splat(int v) { return ((uint32_t)v & 0xffffu) * 0x10001u; }
// bit r <- bit 15 of f_r, bit r + 4 <- bit 31 of f_r
__device__ __forceinline__ uint32_t x16_gather(uint32_t f0, uint32_t f1, uint32_t f2, uint32_t f3) {
  const uint32_t t = ((f0 >> 15) & 0x10001u) | ((f1 >> 14) & 0x20002u) | ((f2 >> 13) & 0x40004u) |
                     ((f3 >> 12) & 0x80008u);
  return (t & 0xfu) | ((t >> 12) & 0xf0u);
}
__device__ __forceinline__ int x16_lo(uint32_t x) { return (int)(int16_t)(x & 0xffffu); }
__device__ __forceinline__ int x16_hi(uint32_t x) { return (int)(int16_t)(x >> 16); }

// register view of the slots one below for register (g, 0) of a thread with G
// groups: the low half is slot 8g - 1 (the high half of group g - 1's register
// 3, or of the previous thread's last register, pv), the high half slot 8g + 3
template <int G>
__device__ __forceinline__ uint32_t x16_down_g(const uint32_t (&X)[4 * G], int g, uint32_t pv) {
  return x16_down0(X[4 * g + 3], g ? X[g ? 4 * g - 1 : 0] : pv);
}
// register view of the slots one above for register (g, 3): slot 8g + 4 (high
// half of register (g, 0)) and slot 8g + 8 (low half of group g + 1's register
// 0, or of the next thread's first register, nx)
template <int G>
__device__ __forceinline__ uint32_t x16_up_g(const uint32_t (&X)[4 * G], int g, uint32_t nx) {
  return x16_up3(X[4 * g], g < G - 1 ? X[g < G - 1 ? 4 * g + 4 : 0] : nx);
}

// the raw update of the 8G cells of one thread on one antidiagonal.  Register
// 4g + r holds slot 8g + r (low half) and slot 8g + r + 4 (high half), so each
// group of four registers is laid out as a thread of eight slots, and its
// traceback flags form word g of the thread (nib[g]).
template <int G, bool LOCAL, bool TB, int DELTA, int DOFF>
__device__ __forceinline__ void x16_cells(const uint32_t (&H1)[4 * G], const uint32_t (&E1)[4 * G],
                                          const uint32_t (&F1)[4 * G], const uint32_t (&H2)[4 * G],
                                          uint32_t pvH1, uint32_t pvE1, uint32_t pvH2, uint32_t nxH1,
                                          uint32_t nxF1, uint32_t nxH2, const uint32_t (&s2)[4 * G],
                                          uint32_t NOE2, uint32_t NE2, uint32_t Z2, uint32_t (&Hr)[4 * G],
                                          uint32_t (&Er)[4 * G], uint32_t (&Fr)[4 * G], uint32_t (&nib)[G]) {
  uint32_t fl[4 * G][4];  // traceback flags of each register: F extended, E extended, F > max(D, E), E > D
#pragma unroll
  for (int g = 0; g < G; ++g) {
  uint32_t acc = 0;
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    // registers in the order 0, 2, 1, 3: the flags of r and r + 2 pack together
    const int rq = (rr & 1) * 2 + (rr >> 1), r = 4 * g + rq;
    // left (slot - 1 + delta) and up (slot + delta) on k-1, diagonal on k-2
    const uint32_t Hl = DELTA ? H1[r] : (rq ? H1[rq ? r - 1 : 0] : x16_down_g<G>(H1, g, pvH1));
    const uint32_t El = DELTA ? E1[r] : (rq ? E1[rq ? r - 1 : 0] : x16_down_g<G>(E1, g, pvE1));
    const uint32_t Hu = DELTA ? (rq < 3 ? H1[rq < 3 ? r + 1 : 0] : x16_up_g<G>(H1, g, nxH1)) : H1[r];
    const uint32_t Fu = DELTA ? (rq < 3 ? F1[rq < 3 ? r + 1 : 0] : x16_up_g<G>(F1, g, nxF1)) : F1[r];
    uint32_t Hd;
    if (DOFF == 0)
      Hd = H2[r];
    else if (DOFF < 0)
      Hd = rq ? H2[rq ? r - 1 : 0] : x16_down_g<G>(H2, g, pvH2);
    else
      Hd = rq < 3 ? H2[rq < 3 ? r + 1 : 0] : x16_up_g<G>(H2, g, nxH2);
    const uint32_t D = __viaddmax_s16x2_relu(Hd, s2[r], 0u);
    const uint32_t Hol = __viaddmax_s16x2_relu(Hl, NOE2, 0u);
    const uint32_t E = __viaddmax_s16x2(El, NE2, Hol);
    const uint32_t Hou = __viaddmax_s16x2_relu(Hu, NOE2, 0u);
    const uint32_t F = __viaddmax_s16x2(Fu, NE2, Hou);
    const uint32_t DE = __vimax_s16x2_relu(D, E);
    const uint32_t H = LOCAL ? __vimax3_s16x2_relu(DE, F, Z2) : __vimax_s16x2_relu(DE, F);
    Hr[r] = H;
    Er[r] = E;
    Fr[r] = F;
    if (TB) {
      // nibble bits c: 3 E > D, 2 F > max(D, E), 1 E extended, 0 F extended.
      // The flag of slot r (bit 15 of its difference) belongs at bit
      // 28 - 4r + c of the word, that of slot r + 4 (bit 31) at 12 - 4r + c.
      // Registers r and r + 2 place a flag 8 bits apart, so one byte permute
      // takes the four sign bits of flag c of both registers as 0x00 / 0xff
      // bytes (255 x flag) in the order of their target bits, and a
      // multiply-add by 2^(4 - 4r + c) on the FMA pipe adds 255 x those bits to
      // a sum.  The sum is 255 x the word; 255 is odd, so one multiply by its
      // inverse mod 2^32 gives the word.
      fl[r][3] = x16_gt(E, D);
      fl[r][2] = x16_gt(F, DE);
      fl[r][1] = x16_gt(E, Hol);
      fl[r][0] = x16_gt(F, Hou);
      if (rq >= 2) {
#pragma unroll
        for (int c = 3; c >= 0; --c) {
          uint32_t pk;
          asm("prmt.b32 %0, %1, %2, 0xD9FB;" : "=r"(pk) : "r"(fl[r][c]), "r"(fl[r - 2][c]));
          asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(acc) : "r"(pk), "r"(1u << (4 - 4 * (rq - 2) + c)), "r"(acc));
        }
      }
    }
  }
  if (TB) nib[g] = acc * 0xfefefeffu;  // 255^-1 mod 2^32
  }
}

// runtime knobs of the packed sweep (a test hook can switch rebasing off, so
// that long pairs leave the 16-bit range and take the int32 rerun)
struct X16Knobs {
  int rebase;  // distance of the best from C0 that moves the base; <= 0: never
};

#ifndef FILTR_X16_MINB
#define FILTR_X16_MINB 1
#endif
// UNI: one match and one mismatch score (codes compared), else a score table
// G: groups of four registers (eight slots) per thread -- 1, or 2 for a one-warp
// group holding a 512-slot window (W = 1 only)
template <int W, int G, bool LOCAL, bool TB, bool ZD, bool UNI>
// (16-slot threads: at most 168 registers, three blocks of four groups per SM)
__global__ void __launch_bounds__(W == 1 ? 128 : W * 32, W == 1 ? (G == 2 ? 3 : FILTR_X16_MINB) : 1)
    k_xdrop16(const FullArgs a, uint32_t *overflow, uint32_t *n_overflow, X16Knobs kn) {
  static_assert(G == 1 || (G == 2 && W == 1), "16 slots per thread in one-warp groups only");
  constexpr int S = 8 * G, P = 4 * G;
  constexpr int WCODE = W * G;  // the group width the host and the walks know: slots / 256
  constexpr int WIN = W * 32 * S;
  constexpr int GROUPS = (W == 1) ? 4 : 1;
  __shared__ X16Shared<W> shm[GROUPS];
  __shared__ int8_t s_sub[MAX_ALPHA * MAX_ALPHA];
  const int A = a.sp.alphabet;
  for (int t = threadIdx.x; t < A * A; t += blockDim.x) s_sub[t] = a.sp.subst[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (W == 1) ? 0 : (int)(threadIdx.x >> 5);
  const int grp = (W == 1) ? (int)(threadIdx.x >> 5) : 0;
  X16Shared<W> &sh = shm[grp];
  const int tid = warp * 32 + lane;
  const int base_slot = tid * S;
  const int o = a.sp.o, e = a.sp.e, oe = o + e;
  const int X = a.sp.xdrop;
  const int smax = max(a.sp.smax, 0);
  // the largest packed best that leaves every formed value inside 16 bits,
  // and the lowest threshold that keeps every relevant value above the floor
  const int pceil = 0x7fff - 4 * smax - 2 * oe - 8;
  const int pfloor = 2 * smax + 2 * oe + 8;
  const uint32_t MA2 = x16_splat(a.sp.uni_match), MI2 = x16_splat(a.sp.uni_mismatch);
  const uint32_t NOE2 = x16_splat(-oe), NE2 = x16_splat(-e);

  auto gsync = [&]() {
    if (W == 1)
      __syncwarp();
    else
      __syncthreads();
  };

  bool first_item = true;
  for (;;) {
    // ---- next pair ------------------------------------------------------------
    uint32_t t0 = 0;
    if (a.ck) {
      t0 = (first_item && grp == 0) ? 0u : a.n_order;
      first_item = false;
    } else if (W == 1) {
      if (lane == 0) t0 = atomicAdd(a.counter, 1u);
      t0 = __shfl_sync(X16_FULL, t0, 0);
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
    const uint8_t *rs = a.b.r_seq + a.b.r_off[p];
    int64_t blo = -(int64_t)M, bhi = N;
    if (a.sp.use_band) band_limits(M, N, a.sp.band, a.sp.band_literal, &blo, &bhi);
    const int band_lo = (int)max(blo, -(int64_t)M), band_hi = (int)min(bhi, (int64_t)N);

    const XdCkpt *ck = a.ck;
    const int ckmode = ck ? ck->mode : 0;
    const int seg = ck ? ck->k_start / ck->C : 0;
    if (ckmode == 3) {
      bool skip = ck->flags[0] != 0 || ck->flags[1 + seg] != 0;
      if (!skip && ck->k_start > 0)
        skip = ck->buf[(int64_t)seg * xd_ckpt_stride() + XCK_USED] > WIN;
      if (skip) break;
    }
    uint32_t *tbp = nullptr;
    int32_t *ckp = nullptr;
    unsigned long long rsv = 0;
    if (TB) {
      if (ckmode == 2) {
        ckp = ck->seg_ck;
        tbp = ck->seg_tb;
      } else if (ckmode == 3) {
        const unsigned long long need = (unsigned long long)ck->C * (WIN / 8);
        if (W == 1) {
          if (lane == 0) rsv = atomicAdd(ck->pool_next, need);
          rsv = __shfl_sync(X16_FULL, rsv, 0);
        } else {
          if (threadIdx.x == 0) sh.rsv = atomicAdd(ck->pool_next, need);
          __syncthreads();
          rsv = sh.rsv;
          __syncthreads();
        }
        if (rsv + need > ck->pool_words) {
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

    // ---- antidiagonal 0 (or the checkpoint resumed) ----------------------------
    uint32_t H1[P], E1[P], F1[P], H2[P];
#pragma unroll
    for (int r = 0; r < P; ++r) H1[r] = E1[r] = F1[r] = H2[r] = 0u;
    int base = 0;  // real value of packed C0
    if (tid == 0) H1[0] = (uint32_t)X16_C0;  // H(0, 0) = 0
    int c = 0, dprev = 0;
    int best = 0, lo = 0, hi = 0, dbest = 0;
    int bv = 0, bi = 0, bj = 0;  // best cell so far (group-uniform)
    uint64_t cells = 0;
    int status = FILTR_ST_OK;
    bool corner = false;
    int cornerH = INT_MIN;
    if (TB && tid == 0 && ckmode == 0) ckp[0] = 0;
    int k_first = 1, k_last = M + N;
    int row0 = 0;  // traceback row of antidiagonal k: k - row0
    if (ckmode >= 2) {
      k_first = ck->k_start + 1;
      row0 = k_first;
      k_last = min(ck->k_end, M + N);
      if (ck->k_start > 0) {
        const int32_t *rec = ck->buf + (int64_t)seg * xd_ckpt_stride();
        c = rec[XCK_ORIGIN];
        dprev = rec[XCK_DPREV];
        best = rec[XCK_BEST];
        lo = rec[XCK_LO];
        hi = rec[XCK_HI];
        dbest = rec[XCK_DBEST];
        base = rec[XCK_BEST];
        const int wwin = rec[XCK_WIN];
        auto pk = [&](int v) -> uint32_t {  // real -> packed (minus infinity and far below: 0)
          const int x = v - base + X16_C0;
          return (v <= NEG_HALF || x <= 0) ? 0u : (uint32_t)min(x, 0x7fff);
        };
        // records hold eight-slot threads: group g of this thread is record thread tid * G + g
#pragma unroll
        for (int r = 0; r < P; ++r) {
          const int g = r >> 2, rq = r & 3;
          const int32_t *mine = rec + XCK_HDR + (tid * G + g) * 32;
          const bool inl = base_slot + 8 * g + rq < wwin, inh = base_slot + 8 * g + rq + 4 < wwin;
          H1[r] = (inl ? pk(mine[rq]) : 0u) | ((inh ? pk(mine[rq + 4]) : 0u) << 16);
          E1[r] = (inl ? pk(mine[8 + rq]) : 0u) | ((inh ? pk(mine[8 + rq + 4]) : 0u) << 16);
          F1[r] = (inl ? pk(mine[16 + rq]) : 0u) | ((inh ? pk(mine[16 + rq + 4]) : 0u) << 16);
          H2[r] = (inl ? pk(mine[24 + rq]) : 0u) | ((inh ? pk(mine[24 + rq + 4]) : 0u) << 16);
        }
        if (ckmode == 3) {
          bv = rec[XCK_BV];
          bi = rec[XCK_BI];
          bj = rec[XCK_BJ];
          cells = (uint64_t)(uint32_t)rec[XCK_CELLS_LO] | ((uint64_t)(uint32_t)rec[XCK_CELLS_HI] << 32);
        }
      }
    }
    int brun = best;  // running best (FILTR_PRUNE_XDROP_RUNNING); best is antidiagonal k-1's
    // the best cell is the result of local alignments; Z-drop needs each
    // antidiagonal's best diagonal.  A global X-drop pair reports its best
    // cell only when it is dropped, which it then takes from the int32 rerun,
    // so its sweep keeps neither.
    const bool track = (LOCAL || ZD) && ckmode != 2;
    const bool need_bs = ZD || track;
    bool ended = false;
    if (W > 1) {
      const int b0 = (k_first - 1) & 1;
      if (lane == 0) sh.first[b0][warp] = Edge16{H1[0], E1[0], F1[0], H2[0]};
      if (lane == 31) sh.last[b0][warp] = Edge16{H1[P - 1], E1[P - 1], F1[P - 1], H2[P - 1]};
      __syncthreads();
    }
    // window origin and codes of k_first: the exact left end of its range
    auto range_lo = [&](int kk, int dl) {  // first column of antidiagonal kk with d >= dl
      return max(max(0, kk - M), (kk + max(dl, band_lo) + 1) >> 1);
    };
    int cn = min(range_lo(k_first, lo - 1), c + 1);
    uint32_t qh[P], rh[P];  // residue codes of register (g, r): slots 8g + r and 8g + r + 4
#pragma unroll
    for (int r = 0; r < P; ++r) {
      uint32_t qv = 0, rv = 0;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int pp = base_slot + 8 * (r >> 2) + (r & 3) + 4 * hh;
        const int j = cn + pp, i = k_first - j;
        const uint32_t qc = (i >= 1 && i <= M) ? q[i - 1] : 0u;
        const uint32_t rc = (j >= 1 && j <= N) ? rs[j - 1] : 0u;
        qv |= qc << (16 * hh);
        rv |= rc << (16 * hh);
      }
      qh[r] = qv;
      rh[r] = rv;
    }
    uint32_t nextc = 0;  // the code entering the window at the next antidiagonal
    // reductions of the last antidiagonal masked (consumed one antidiagonal later)
    bool pending = false;
    int pmax = 0, plo = INT_MAX, phi = INT_MIN, pbs = -1;  // of antidiagonal k - 1, origin c
    int k = k_first;

    // consume the reductions of antidiagonal kk (origin ckk): best, live range,
    // best cell; returns false when nothing was alive on kk
    auto consume = [&](int kk, int ckk, int gmax, int glo, int ghi, int gbs) -> bool {
      if (glo == INT_MAX) return false;
      const int gv = gmax - X16_C0 + base;
      const int jj = ckk + gbs, ii = kk - jj;
      if (track && (gv > bv || (gv == bv && (ii < bi || (ii == bi && jj < bj))))) {
        bv = gv;
        bi = ii;
        bj = jj;
      }
      best = gv;
      if (!a.sp.xrun || gv > brun) {
        brun = gv;
        if (ZD) dbest = 2 * jj - kk;
      }
      lo = 2 * (ckk + glo) - kk;
      hi = 2 * (ckk + ghi) - kk;
      if (kk == M + N) corner = true;
      return true;
    };

    for (; k <= k_last; ++k) {
      const int delta = cn - c;
      // ---- codes at the new origin --------------------------------------------
      if (k != k_first) {
        if (delta == 1) {  // reference codes move down one slot, the new one enters slot S - 1
#pragma unroll
          for (int g = 0; g < G; ++g) {
            // slot 8g + 8 enters group g from the next group (or is the new code)
            const uint32_t in = g < G - 1 ? (rh[g < G - 1 ? 4 * g + 4 : 0] & 0xffffu) : nextc;
            const uint32_t t = (rh[4 * g] >> 16) | (in << 16);
            rh[4 * g] = rh[4 * g + 1];
            rh[4 * g + 1] = rh[4 * g + 2];
            rh[4 * g + 2] = rh[4 * g + 3];
            rh[4 * g + 3] = t;
          }
        } else {  // query codes move up one slot, the new one enters slot 0
#pragma unroll
          for (int g = G - 1; g >= 0; --g) {
            // slot 8g - 1 enters group g from the group before (or is the new code)
            const uint32_t in = g ? (qh[g ? 4 * g - 1 : 0] >> 16) : nextc;
            const uint32_t t = in | (qh[4 * g + 3] << 16);
            qh[4 * g + 3] = qh[4 * g + 2];
            qh[4 * g + 2] = qh[4 * g + 1];
            qh[4 * g + 1] = qh[4 * g];
            qh[4 * g] = t;
          }
        }
      }
      // ---- substitution scores of the eight cells --------------------------------
      uint32_t s2[P];
      if (UNI) {
#pragma unroll
        for (int r = 0; r < P; ++r) {
          const uint32_t ne = x16_halfmask((qh[r] ^ rh[r]) + 0x7fff7fffu);  // codes differ
          s2[r] = (ne & MI2) | (~ne & MA2);
        }
      } else {
#pragma unroll
        for (int r = 0; r < P; ++r) {
          const uint32_t idx = qh[r] * (uint32_t)A + rh[r];
          const int slo = s_sub[idx & 0xffffu], shi = s_sub[idx >> 16];
          s2[r] = ((uint32_t)slo & 0xffffu) | ((uint32_t)shi << 16);
        }
      }
      // ---- neighbour values across thread boundaries -----------------------------
      const int buf = (k - 1) & 1;
      uint32_t pvH1 = 0, pvE1 = 0, pvH2 = 0, nxH1 = 0, nxF1 = 0, nxH2 = 0;
      const int doff = delta + dprev - 1;
      if (delta == 0) {
        pvH1 = __shfl_up_sync(X16_FULL, H1[P - 1], 1);
        pvE1 = __shfl_up_sync(X16_FULL, E1[P - 1], 1);
        if (lane == 0) {
          const bool in = W > 1 && warp > 0;
          pvH1 = in ? sh.last[buf][in ? warp - 1 : 0].H1 : 0u;
          pvE1 = in ? sh.last[buf][in ? warp - 1 : 0].E1 : 0u;
        }
      } else {
        nxH1 = __shfl_down_sync(X16_FULL, H1[0], 1);
        nxF1 = __shfl_down_sync(X16_FULL, F1[0], 1);
        if (lane == 31) {
          const bool in = W > 1 && warp < W - 1;
          nxH1 = in ? sh.first[buf][in ? warp + 1 : 0].H1 : 0u;
          nxF1 = in ? sh.first[buf][in ? warp + 1 : 0].F1 : 0u;
        }
      }
      if (doff < 0) {
        pvH2 = __shfl_up_sync(X16_FULL, H2[P - 1], 1);
        if (lane == 0) pvH2 = (W > 1 && warp > 0) ? sh.last[buf][warp > 0 ? warp - 1 : 0].H2 : 0u;
      } else if (doff > 0) {
        nxH2 = __shfl_down_sync(X16_FULL, H2[0], 1);
        if (lane == 31) nxH2 = (W > 1 && warp < W - 1) ? sh.first[buf][warp < W - 1 ? warp + 1 : 0].H2 : 0u;
      }
      // ---- raw cells of k ------------------------------------------------------
      const uint32_t Z2 = LOCAL ? x16_splat(min(max(X16_C0 - base, 0), 0x7fff)) : 0u;
      uint32_t Hr[P], Er[P], Fr[P];
      uint32_t nib[G];
      if (delta == 1) {
        if (doff == 0)
          x16_cells<G, LOCAL, TB, 1, 0>(H1, E1, F1, H2, pvH1, pvE1, pvH2, nxH1, nxF1, nxH2, s2, NOE2, NE2, Z2, Hr,
                                     Er, Fr, nib);
        else
          x16_cells<G, LOCAL, TB, 1, 1>(H1, E1, F1, H2, pvH1, pvE1, pvH2, nxH1, nxF1, nxH2, s2, NOE2, NE2, Z2, Hr,
                                     Er, Fr, nib);
      } else {
        if (doff == 0)
          x16_cells<G, LOCAL, TB, 0, 0>(H1, E1, F1, H2, pvH1, pvE1, pvH2, nxH1, nxF1, nxH2, s2, NOE2, NE2, Z2, Hr,
                                     Er, Fr, nib);
        else
          x16_cells<G, LOCAL, TB, 0, -1>(H1, E1, F1, H2, pvH1, pvE1, pvH2, nxH1, nxF1, nxH2, s2, NOE2, NE2, Z2,
                                      Hr, Er, Fr, nib);
      }

      // ---- the reductions of k - 1 -------------------------------------------------
      if (pending) {
        int gmax = pmax, glo = plo, ghi = phi, gbs = pbs;
        if (W > 1) {
          const int nb = (k - 1) & 1;
          const int v0 = lane < W ? sh.red[nb][lane][0] : INT_MIN;
          gmax = __reduce_max_sync(X16_FULL, v0);
          glo = __reduce_min_sync(X16_FULL, lane < W ? sh.red[nb][lane][1] : INT_MAX);
          ghi = __reduce_max_sync(X16_FULL, lane < W ? sh.red[nb][lane][2] : INT_MIN);
          gbs = __reduce_max_sync(X16_FULL, (lane < W && v0 == gmax) ? sh.red[nb][lane][3] : -1);
        }
        pending = false;
        if (!consume(k - 1, c, gmax, glo, ghi, gbs)) {  // nothing alive on k - 1: the sweep ends there
          ended = true;
          break;
        }
        // keep the packed range centred on the best
        const int bp = best - base + X16_C0;
        if (kn.rebase > 0 && (bp > X16_C0 + kn.rebase || bp < X16_C0 - kn.rebase)) {
          const int sft = bp - X16_C0;
          base += sft;
          const uint32_t d2 = x16_splat(-sft);
#pragma unroll
          for (int r = 0; r < P; ++r) {
            H1[r] = __viaddmax_s16x2_relu(H1[r], d2, 0u);
            E1[r] = __viaddmax_s16x2_relu(E1[r], d2, 0u);
            F1[r] = __viaddmax_s16x2_relu(F1[r], d2, 0u);
            H2[r] = __viaddmax_s16x2_relu(H2[r], d2, 0u);
            Hr[r] = __viaddmax_s16x2_relu(Hr[r], d2, 0u);
            Er[r] = __viaddmax_s16x2_relu(Er[r], d2, 0u);
            Fr[r] = __viaddmax_s16x2_relu(Fr[r], d2, 0u);
          }
        }
      }
      // ---- candidate range of k, window check, next origin ---------------------------
      const int dl = max(lo - 1, band_lo), dh = min(hi + 1, band_hi);
      const int jA = max(max(0, k - M), (k + dl + 1) >> 1);
      const int jB = min(min(N, k), (k + dh) >> 1);
      if (jA > jB) {
        ended = true;
        break;
      }
      if (jB - cn + 1 > WIN) {
        status = FILTR_ST_TOO_WIDE;
        break;
      }
      // thresholds of k, and the range checks of the packed form
      const int bref = a.sp.xrun ? brun : best;
      const int bpp = best - base + X16_C0;   // packed best of k - 1
      const int rpp = bref - base + X16_C0;   // packed reference of the threshold
      int thr = rpp - X;
      int tmin = thr;
      if (ZD) {
        const int da = 2 * jA - k - dbest, db = 2 * jB - k - dbest;
        tmin = thr - max(abs(da), abs(db));
      }
      if (bpp > pceil || tmin < pfloor) {
        status = X16_OVERFLOW;
        break;
      }
      thr = min(thr, 0x7fff);
      {  // the next antidiagonal's origin (a lower bound of its range's left end) and code
        const int cnx = min(range_lo(k + 1, lo - 2), cn + 1);
        if (k < k_last) {  // a reference code if the origin moves, else a query code
          const bool mvx = cnx - cn == 1;
          const int j = cnx + base_slot + S - 1, i = k + 1 - cnx - base_slot;
          const bool ok = mvx ? (j >= 1 && j <= N) : (i >= 1 && i <= M);
          const uint8_t *src = mvx ? rs + (j - 1) : q + (i - 1);
          nextc = ok ? *src : 0u;
        }
        // ---- prune k --------------------------------------------------------------
        const int vA = jA - cn - base_slot, vB = jB - cn - base_slot;
        constexpr uint32_t SFULL = (1u << S) - 1u;
        uint32_t dom = 0;  // bit s: slot s of the thread is in the candidate range
        if (vB >= 0 && vA < S) dom = (SFULL << max(vA, 0)) & (SFULL >> (S - 1 - min(vB, S - 1))) & SFULL;
        const int zx = ZD ? 2 * (cn + base_slot) - k - dbest : 0;
        uint32_t t2 = 0, am = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          // the group's range bits: slot 8g + r at bit r, slot 8g + r + 4 at bit 16 + r
          const uint32_t dsp = ((dom >> (8 * g)) & 0xfu) | (((dom >> (8 * g + 4)) & 0xfu) << 16);
          uint32_t amw = 0;
#pragma unroll
          for (int rq = 0; rq < 4; ++rq) {
            const int r = 4 * g + rq;
            uint32_t th2;
            if (ZD) {
              const int tl = min(max(thr - abs(zx + 2 * (8 * g + rq)), 1), 0x7fff);
              const int tu = min(max(thr - abs(zx + 2 * (8 * g + rq) + 8), 1), 0x7fff);
              th2 = (uint32_t)tl | ((uint32_t)tu << 16);
            } else {
              th2 = x16_splat(thr);
            }
            // [H >= threshold] per half, kept only inside the candidate range
            const uint32_t m = x16_halfmask(x16_ge(Hr[r], th2) & (dsp << (15 - rq)));
            H2[r] = H1[r];
            H1[r] = Hr[r] & m;
            E1[r] = Er[r] & m;
            F1[r] = Fr[r] & m;
            t2 = __vimax_s16x2_relu(t2, H1[r]);
            amw |= m & (0x10001u << rq);  // live slots: bit rq (low half), bit 16 + rq (high half)
          }
          am |= ((amw & 0xfu) | ((amw >> 12) & 0xf0u)) << (8 * g);
        }
        const int tmax = max(x16_lo(t2), x16_hi(t2));
        const int tl = am ? __ffs(am) - 1 : -1;
        const int th = am ? 31 - __clz(am) : -1;
        // the largest live slot holding the thread's maximum (smallest i)
        int ts = -1;
        if (need_bs) {
          const uint32_t tm2 = x16_splat(tmax);
          uint32_t bm = 0;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            uint32_t bmw = 0;
#pragma unroll
            for (int rq = 0; rq < 4; ++rq)
              bmw |= x16_halfmask(x16_ge(H1[4 * g + rq], tm2)) & (0x10001u << rq);
            bm |= ((bmw & 0xfu) | ((bmw >> 12) & 0xf0u)) << (8 * g);
          }
          bm &= am;
          ts = bm ? 31 - __clz(bm) : -1;
        }
        // ---- traceback word and origin of k -----------------------------------------
        if (TB) {
          const int64_t row = (int64_t)(k - row0);
          // only the 32-byte sectors (8 / G threads) holding a slot of the range
          constexpr int TPS = 8 / G;
          const unsigned act = __ballot_sync(X16_FULL, dom != 0);
          if ((act >> (lane & (32 - TPS))) & ((1u << TPS) - 1u)) {
#pragma unroll
            for (int g = 0; g < G; ++g) tbp[row * (WIN / 8) + G * tid + g] = nib[g];
          }
          if (tid == 0) ckp[row] = cn;
        }
        {
          const int a0 = max(jA, 1), b0 = min(jB, k - 1);
          cells += (uint64_t)max(b0 - a0 + 1, 0);
        }
        if (k == M + N) {  // the corner is the single cell of antidiagonal M + N
          const int pcn = N - cn - base_slot;
          if (pcn >= 0 && pcn < S) {
            // slot pcn: register 4 (pcn / 8) + pcn % 4, high half when pcn % 8 >= 4
            uint32_t hv = 0;
#pragma unroll
            for (int r = 0; r < P; ++r)
              if (4 * (pcn >> 3) + (pcn & 3) == r) hv = H1[r];
            const int v = ((pcn & 7) < 4) ? (int)(hv & 0xffffu) : (int)(hv >> 16);
            cornerH = v ? v - X16_C0 + base : NEG;
          }
        }
        // ---- reductions of k (consumed after the next raw update) --------------------
        const int wmax = __reduce_max_sync(X16_FULL, am ? tmax : 0);
        const int wlo = __reduce_min_sync(X16_FULL, am ? base_slot + tl : INT_MAX);
        const int whi = __reduce_max_sync(X16_FULL, am ? base_slot + th : INT_MIN);
        const int wbs = need_bs ? __reduce_max_sync(X16_FULL, (am && tmax == wmax) ? base_slot + ts : -1) : 0;
        pmax = wmax;
        plo = wlo;
        phi = whi;
        pbs = wbs;
        pending = true;
        if (W > 1) {
          const int nb = k & 1;
          if (lane == 0) {
            sh.red[nb][warp][0] = wlo == INT_MAX ? INT_MIN : wmax;
            sh.red[nb][warp][1] = wlo;
            sh.red[nb][warp][2] = whi;
            sh.red[nb][warp][3] = wbs;
            sh.first[nb][warp] = Edge16{H1[0], E1[0], F1[0], H2[0]};
          }
          if (lane == 31) sh.last[nb][warp] = Edge16{H1[P - 1], E1[P - 1], F1[P - 1], H2[P - 1]};
          __syncthreads();
        }
        c = cn;
        dprev = delta;
        cn = cnx;
      }
    }
    if (pending) {  // the last antidiagonal's reductions
      int gmax = pmax, glo = plo, ghi = phi, gbs = pbs;
      if (W > 1) {
        const int nb = (k - 1) & 1;
        const int v0 = lane < W ? sh.red[nb][lane][0] : INT_MIN;
        gmax = __reduce_max_sync(X16_FULL, v0);
        glo = __reduce_min_sync(X16_FULL, lane < W ? sh.red[nb][lane][1] : INT_MAX);
        ghi = __reduce_max_sync(X16_FULL, lane < W ? sh.red[nb][lane][2] : INT_MIN);
        gbs = __reduce_max_sync(X16_FULL, (lane < W && v0 == gmax) ? sh.red[nb][lane][3] : -1);
      }
      pending = false;
      if (!consume(k - 1, c, gmax, glo, ghi, gbs)) ended = true;
    }
    if (status == FILTR_ST_OK && k > k_last && k_last == M + N) ended = true;
    // a dropped global pair without its best cell: the int32 sweep finds it
    if (!LOCAL && !track && ckmode != 2 && status == FILTR_ST_OK && ended && !corner) status = X16_OVERFLOW;
    if (ckmode == 3 && status == FILTR_ST_TOO_WIDE && WCODE < XD_MAX_WARPS) break;
    if (ckmode >= 2 && status == X16_OVERFLOW) {  // the whole pair goes to the int32 sweep
      if (tid == 0 && ckmode == 3) ck->flags[0] = 3;
      break;
    }

    // the corner value lives in one thread; broadcast it
    if (!LOCAL) {
      int ch = __reduce_max_sync(X16_FULL, cornerH);
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
      int used = 0;
#pragma unroll
      for (int r = 0; r < P; ++r) {
        const int sl = base_slot + 8 * (r >> 2) + (r & 3);  // slot of the low half
        if ((H1[r] | E1[r] | F1[r] | H2[r]) & 0xffffu) used = max(used, sl + 1);
        if ((H1[r] | E1[r] | F1[r] | H2[r]) >> 16) used = max(used, sl + 5);
      }
      used = __reduce_max_sync(X16_FULL, used);
      if (W > 1) {
        __syncthreads();
        if (lane == 0) sh.red[0][warp][0] = used;
        __syncthreads();
        for (int w = 0; w < W; ++w) used = max(used, sh.red[0][w][0]);
      }
      auto rv = [&](uint32_t x, int hh) -> int32_t {  // packed half -> real (0: minus infinity)
        const int v = hh ? (int)(x >> 16) : (int)(x & 0xffffu);
        return v ? v - X16_C0 + base : NEG;
      };
      // eight-slot record threads: group g of this thread is record thread tid * G + g
#pragma unroll
      for (int r = 0; r < P; ++r) {
        int32_t *mine = rec + XCK_HDR + (tid * G + (r >> 2)) * 32;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int s = (r & 3) + 4 * hh;
          mine[s] = rv(H1[r], hh);
          mine[8 + s] = rv(E1[r], hh);
          mine[16 + s] = rv(F1[r], hh);
          mine[24 + s] = rv(H2[r], hh);
        }
      }
      if (tid == 0) {
        rec[XCK_ORIGIN] = c;
        rec[XCK_DPREV] = dprev;
        rec[XCK_BEST] = a.sp.xrun ? brun : best;
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
          ck->seg_w[seg] = WCODE;
        }
        ck->flags[1 + seg] = WCODE;
      }
      gsync();
      continue;
    }
    if (tid == 0 && ckmode != 2) {
      if (ckmode == 3) {
        if (TB && status != FILTR_ST_TOO_WIDE) {
          ck->seg_off[seg] = rsv;
          ck->seg_w[seg] = WCODE;
        }
        ck->flags[0] = 1;
        if (status != FILTR_ST_TOO_WIDE) ck->flags[1 + seg] = WCODE;
      }
      int score = 0, ei = 0, ej = 0;
      if (status == FILTR_ST_TOO_WIDE) {
        const uint32_t slot = atomicAdd(n_overflow, 1u);
        overflow[slot] = p;
      } else if (status == X16_OVERFLOW) {
        const uint32_t slot = atomicAdd(a.n_ovf16, 1u);
        a.ovf16[slot] = p;
        status = FILTR_ST_TOO_WIDE;  // until the int32 rerun writes the result
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

// Group widths: W = 1 (256 slots) runs one warp per pair (8 slots per thread,
// four pairs per 128-thread block).  W = 2 (512 slots) runs one warp of 16-slot
// threads for batched pairs, where the bookkeeping done once per warp and the
// absence of block barriers pay, and two warps of 8-slot threads for the
// segments of one long pair (a.ck), where the shorter chain of two half-loaded
// warps gives the lower latency per antidiagonal.  The traceback rows and the
// checkpoint records of W = 2 are the same in either form: thread t of the
// one-warp group writes words 2t and 2t + 1.  W >= 4 runs W warps of 8-slot
// threads.
template <int KW, int G, bool LOCAL, bool TB, bool ZD>
cudaError_t x16_launch(const FullArgs &a, int grid, uint32_t *ovf, uint32_t *novf, X16Knobs kn,
                       cudaStream_t s) {
  if (a.sp.uni)
    k_xdrop16<KW, G, LOCAL, TB, ZD, true><<<grid, KW == 1 ? 128 : KW * 32, 0, s>>>(a, ovf, novf, kn);
  else
    k_xdrop16<KW, G, LOCAL, TB, ZD, false><<<grid, KW == 1 ? 128 : KW * 32, 0, s>>>(a, ovf, novf, kn);
  return cudaGetLastError();
}

template <int KW, int G, bool ZD>
cudaError_t x16_dispatch(const FullArgs &a, int grid, uint32_t *ovf, uint32_t *novf, X16Knobs kn,
                         cudaStream_t s) {
  const bool L = a.sp.mode == FILTR_LOCAL, T = a.sp.traceback != 0;
  if (L) return T ? x16_launch<KW, G, true, true, ZD>(a, grid, ovf, novf, kn, s)
                  : x16_launch<KW, G, true, false, ZD>(a, grid, ovf, novf, kn, s);
  return T ? x16_launch<KW, G, false, true, ZD>(a, grid, ovf, novf, kn, s)
           : x16_launch<KW, G, false, false, ZD>(a, grid, ovf, novf, kn, s);
}

template <int KW, int G, bool LOCAL, bool TB, bool ZD>
int x16_occ() {
  int nb = 0, nb2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_xdrop16<KW, G, LOCAL, TB, ZD, true>, KW == 1 ? 128 : KW * 32, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_xdrop16<KW, G, LOCAL, TB, ZD, false>, KW == 1 ? 128 : KW * 32,
                                                0);
  return std::min(nb, nb2);
}

template <int KW, int G, bool ZD>
int x16_occ_w(const ScoreParams &sp) {
  const bool L = sp.mode == FILTR_LOCAL, T = sp.traceback != 0;
  if (L) return T ? x16_occ<KW, G, true, true, ZD>() : x16_occ<KW, G, true, false, ZD>();
  return T ? x16_occ<KW, G, false, true, ZD>() : x16_occ<KW, G, false, false, ZD>();
}

template <bool ZD>
cudaError_t x16_launch_any(const FullArgs &a, int W, int grid, uint32_t *ovf, uint32_t *novf, X16Knobs kn,
                           cudaStream_t s) {
  switch (W) {
    case 1: return x16_dispatch<1, 1, ZD>(a, grid, ovf, novf, kn, s);
    case 2: return a.ck ? x16_dispatch<2, 1, ZD>(a, grid, ovf, novf, kn, s)
                        : x16_dispatch<1, 2, ZD>(a, grid, ovf, novf, kn, s);
    case 4: return x16_dispatch<4, 1, ZD>(a, grid, ovf, novf, kn, s);
    case 8: return x16_dispatch<8, 1, ZD>(a, grid, ovf, novf, kn, s);
    case 16: return x16_dispatch<16, 1, ZD>(a, grid, ovf, novf, kn, s);
    case 32: return x16_dispatch<32, 1, ZD>(a, grid, ovf, novf, kn, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool ZD>
int x16_occ_any(int W, const ScoreParams &sp) {
  switch (W) {
    case 1: return x16_occ_w<1, 1, ZD>(sp);
    case 2: return x16_occ_w<1, 2, ZD>(sp);
    case 4: return x16_occ_w<4, 1, ZD>(sp);
    case 8: return x16_occ_w<8, 1, ZD>(sp);
    case 16: return x16_occ_w<16, 1, ZD>(sp);
    case 32: return x16_occ_w<32, 1, ZD>(sp);
    default: return 0;
  }
}

}  // namespace
}  // namespace filtr
