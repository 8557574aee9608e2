// k_pack_impl.cuh -- the batched tiled wavefront with two 16-bit cells per 32-bit
// register (int16x2), for unbanded pairs whose score range fits 15 bits
// (pack_bias).  Results, traceback choices and tie-breaks are those of the
// int32 kernel k_full; only the arithmetic width and the tile layout differ.
//
// Work distribution as in k_full: one warp per pair from a cost-ordered queue,
// the query cut into strips of 32*R rows, lane l owning R rows.  Those R rows
// live in P = R/2 registers: register k holds row k of the lane in its low
// half and row P + k in its high half, and the high half runs one column
// behind the low half, so one instruction updates both:
//   step t, lane l: low half at column cL = 1 + t - 2l, high half at cL - 1.
// Dependencies of register 0 at step t:
//   low half  (row 0, column cL): up and diagonal are lane l-1's last row at
//             columns cL and cL-1, which that lane's high half produced at
//             steps t-1 and t-2 -- one __shfl_up_sync per step carries them;
//   high half (row P, column cL-1): up is this lane's row P-1 at column cL-1,
//             the low half of register P-1 one step ago; diagonal the same
//             two steps ago.
// Registers k > 0 take up and diagonal from register k-1 as in k_full.  A lane
// thus advances two columns of staircase per row of lanes (63 fill steps per
// strip instead of 31).  Steps where some lane has a half outside [1, N] (the
// first 63 and the last 63 of a strip) run a masked copy of the update that
// keeps those halves' state; the others run unmasked.
//
// Values are unsigned 16-bit v + B (B from pack_bias), so additions of signed
// packed constants never carry between halves, max.u16x2 is the signed max,
// and X = A - B + 0x7fff7fff holds [A > B] in bits 15 and 31.  Minus infinity
// (boundary E and F) is e, whose extension e - e = 0 is below every finite
// value.  The query profile in shared memory holds s + 64 (7 bits, 0 for rows
// past M), so one byte permute builds a register's two scores.  Per residue and
// lane it holds the low half's P bytes in PW = ceil(P/4) words, then the high
// half's in another PW, so both halves load as aligned words for every even R.
//
// Traceback, per strip: step-major, then word, then lane; 2G words per lane
// and step (G = ceil(P/8)), word h*G + g holding cells 8g..8g+7 of half h as
// four bit planes -- byte 0: E > D, byte 1: F > max(D, E), byte 2: E took the
// extension, byte 3: F took the extension; bit c of each byte is cell 8g + c.
// The planes are gathered by sign-replicating byte permutes (the two halves'
// sign bits of two differences per permute, each widened to a 0x00 / 0xff
// byte, i.e. 255 x flag) accumulated as sum(permute x 2^c) by multiply-adds on
// the FMA pipe; one multiply by the inverse of 255 mod 2^32 per group of eight
// registers turns the sum into the plane word.
#pragma once

#include <climits>
#include <type_traits>

#include "filtr_internal.h"
#include "plan.h"

namespace filtr {
namespace {

constexpr unsigned PFULL = 0xffffffffu;

template <uint32_t SEL>
__device__ __forceinline__ uint32_t perm(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "n"(SEL));
  return r;
}
__device__ __forceinline__ uint32_t max2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// a + b issued as a multiply-add on the FMA pipe (one == 1 at run time)
__device__ __forceinline__ uint32_t fadd2(uint32_t a, uint32_t b, uint32_t one) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(one), "r"(a));
  return r;
}
// a * b + c on the FMA pipe (low 32 bits)
__device__ __forceinline__ uint32_t fmad32(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
// (x & m) | (y & ~m)
__device__ __forceinline__ uint32_t select_bits(uint32_t m, uint32_t x, uint32_t y) {
  return (x & m) | (y & ~m);
}

template <int B>
struct ScoreSel {  // low half <- byte B of the low word, high half <- byte B of the high word
  static constexpr uint32_t v = B | ((8u | B) << 4) | ((4u + B) << 8) | ((8u | (4u + B)) << 12);
};

// PW words of one half's profile bytes
template <int PW>
struct HalfProf;
template <>
struct HalfProf<1> {
  using T = uint32_t;
};
template <>
struct HalfProf<2> {
  using T = uint2;
};
struct HalfProf3 {
  uint32_t a, b, c;
};
template <>
struct HalfProf<3> {
  using T = HalfProf3;
};
template <>
struct HalfProf<4> {
  using T = uint4;
};

struct PackPair {
  int M, N;
  const uint8_t *q, *r;
  int o, e, A, B;
  uint32_t one;
  const int8_t *s_sub;
  int8_t *prof;
  uint32_t *tb;
};

struct Best {
  int v, i, j;
};
__device__ __forceinline__ void best_put(Best &b, int v, int i, int j) {
  if (v > b.v || (v == b.v && (i < b.i || (i == b.i && j < b.j)))) {
    b.v = v;
    b.i = i;
    b.j = j;
  }
}

template <int R, bool LOCAL, bool AFFINE, bool TB>
__device__ __forceinline__ void pack_strip(const PackPair &PP, int s, int64_t tb_base, int2 *buf,
                                           Best &best, int &endH) {
  constexpr int HS = 32 * R, P = R / 2, G = (P + 7) / 8, WPS = 2 * G;
  constexpr int PW = (P + 3) / 4, PS = pack_prof_stride(R);
  static_assert(R % 2 == 0 && R >= 8 && R <= 32, "packed tile height");
  using HW = typename HalfProf<PW>::T;
  const int lane = threadIdx.x & 31;
  const int M = PP.M, N = PP.N, o = PP.o, e = PP.e, B = PP.B;
  const uint32_t one = PP.one, mone = 0u - PP.one;
  const int oe = AFFINE ? o + e : e;
  const uint32_t MOE = (uint32_t)(-(int64_t)oe * 65537);
  const uint32_t ME = (uint32_t)(-(int64_t)e * 65537);
  // -e in each half for the per-half (DPX) add: ME above is the 32-bit
  // constant, whose high half is -e - 1 to absorb the low half's borrow
  const uint32_t ME16 = ((uint32_t)(-e) & 0xffffu) * 0x10001u;
  const uint32_t K64M = (uint32_t)(-(int64_t)64 * 65537);
  const uint32_t K7F = 0x7fff7fffu;
  const uint32_t K7FME = K7F + ME;
  const uint32_t BZ = (uint32_t)B * 65537u;
  const uint32_t NEG2 = (uint32_t)e * 65537u;
  const int row0 = s * HS;
  const int top = row0 + lane * R + 1;  // first row (1-based) of the lane
  const int nstrips = (M + HS - 1) / HS;

  // query profile of the strip: for residue a, lane l's words at a * PS + 8 PW l
  // hold s(q[row], a) + 64 for its rows top-1 .. top+P-2 (low half), then, PW
  // words later, for rows top+P-1 .. top+R-2 (high half); 0 past M and in the
  // padding bytes of the last word of each half
  {
    int qc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int row = top - 1 + k;
      qc[k] = (row < M) ? (int)PP.q[row] : -1;
    }
    __syncwarp();
    for (int aa = 0; aa < PP.A; ++aa) {
      uint32_t *dst = reinterpret_cast<uint32_t *>(PP.prof + aa * PS + lane * 8 * PW);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int w = 0; w < PW; ++w) {
          uint32_t v = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if (4 * w + b < P) {
              const int c = qc[h * P + 4 * w + b];
              const uint32_t sv = (c >= 0) ? (uint32_t)((int)PP.s_sub[c * PP.A + aa] + 64) : 0u;
              v |= sv << (8 * b);
            }
          }
          dst[h * PW + w] = v;
        }
      }
    }
    __syncwarp();
  }

  // column 0 / row 0: H(0, 0) = 0, H(i, 0) = -(o + i e) (global) or 0 (local),
  // E = minus infinity
  auto h0 = [&](int i) -> uint32_t {
    return (uint32_t)((LOCAL || i == 0) ? B : B - o - i * e) & 0xffffu;
  };
  uint32_t Hc[P], Ec[P], Hm[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    Hc[k] = h0(top + k) | (h0(top + P + k) << 16);
    Ec[k] = NEG2;
    Hm[k] = Hc[k] + MOE;
  }
  // lane 0's view of the row above the strip: H(row0, j), F(row0, j)
  uint32_t prevS = h0(row0) << 16;  // H(row0, 0), the first diagonal
  uint32_t outH = Hc[P - 1], outF = NEG2, Flast = NEG2, hprev = Hc[P - 1];
  const int nsteps = N + 63;
  // best-cell key of the lane so far: a later strip needs a strictly larger H
  uint32_t bestkey = ((uint32_t)(best.v + B) << 16) | 31u;
  int rc_lo = PP.r[0], rc_hi = rc_lo;
  int rc_next = PP.r[min(max(1 - 2 * lane, 1), N) - 1];

  // one step; the steps where some lane has a half outside [1, N] (the first
  // 63 and those from N on) run the masked form, the steady ones the plain
  auto step = [&](const int t, auto edge_tag) {
    constexpr bool EDGE_STEP = decltype(edge_tag)::value;
    const int cL = 1 + t - 2 * lane, cH = cL - 1;
    // steady steps (63 <= t <= N - 1) have every lane's halves inside [1, N]
    const bool actL = !EDGE_STEP || (cL >= 1 && cL <= N);
    const bool actH = !EDGE_STEP || (cH >= 1 && cH <= N);
    uint32_t sH = __shfl_up_sync(PFULL, outH, 1);
    uint32_t sF = __shfl_up_sync(PFULL, outF, 1);
    if (lane == 0) {
      // outside [1, N] the row above is a placeholder, but it must stay inside
      // the biased range: a half that wraps below 0 borrows from (or carries
      // into) the other half of the same register, which at cL = N + 1 is the
      // live cell (i, N) -- H = B (score 0), F = minus infinity keep it in range
      uint32_t hv = (uint32_t)B, fv = (uint32_t)e;
      if (s == 0 && actL) {
        hv = (uint32_t)(LOCAL ? B : B - o - cL * e) & 0xffffu;  // H(0, cL)
      } else if (actL) {
        const int2 v = buf[cL];
        hv = (uint32_t)v.x;
        fv = (uint32_t)v.y;
      }
      sH = hv << 16;
      sF = fv << 16;
    }
    // profile words: low half at column cL, high half at cH (last step's cL)
    rc_hi = rc_lo;
    rc_lo = rc_next;
    rc_next = PP.r[(EDGE_STEP ? min(max(cL + 1, 1), N) : min(cL + 1, N)) - 1];
    const HW wl = *reinterpret_cast<const HW *>(PP.prof + rc_lo * PS + lane * 8 * PW);
    const HW wh = *reinterpret_cast<const HW *>(PP.prof + rc_hi * PS + lane * 8 * PW + 4 * PW);
    const uint32_t *wlw = reinterpret_cast<const uint32_t *>(&wl);
    const uint32_t *whw = reinterpret_cast<const uint32_t *>(&wh);

    uint32_t Hup = perm<0x5432>(sH, Hc[P - 1]);
    uint32_t Fup = perm<0x5432>(sF, Flast);
    uint32_t Hdg = perm<0x5432>(prevS, hprev);
    hprev = Hc[P - 1];
    prevS = sH;
    uint32_t Hmup = fadd2(Hup, MOE, one);
    const uint32_t KM = (actL ? 0x0000ffffu : 0u) | (actH ? 0xffff0000u : 0u);
    uint32_t mkey = 0;  // largest best-cell key of this step (local mode)
    uint32_t accA = 0, accB = 0;
    uint32_t tbw[2 * G > 0 ? 2 * G : 1];

    // the register loop, unmasked for steps where every lane has both halves
    // inside [1, N], masked (inactive halves keep their state) otherwise
    auto regs = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        uint32_t sc;
        switch (k & 3) {
          case 0: sc = perm<ScoreSel<0>::v>(wlw[k >> 2], whw[k >> 2]); break;
          case 1: sc = perm<ScoreSel<1>::v>(wlw[k >> 2], whw[k >> 2]); break;
          case 2: sc = perm<ScoreSel<2>::v>(wlw[k >> 2], whw[k >> 2]); break;
          default: sc = perm<ScoreSel<3>::v>(wlw[k >> 2], whw[k >> 2]); break;
        }
        const uint32_t D = fadd2(Hdg, fadd2(sc, K64M, one), one);
        const uint32_t Hol = Hm[k];
        uint32_t E, F;
        if (AFFINE) {
          // per half max(E_left - e, H_left - (o+e)): one DPX add-max in place of
          // an add and a max, which leaves room on the FMA pipe for X3 below.
          // Signed halves: every biased value is below 0x8000, so the sum
          // stays inside the 16-bit range
          E = __viaddmax_s16x2(Ec[k], ME16, Hol);
          F = __viaddmax_s16x2(Fup, ME16, Hmup);
        } else {
          E = Hol;
          F = Hmup;
        }
        const uint32_t DE = max2(D, E);
        const uint32_t H = LOCAL ? __vimax3_u16x2(DE, F, BZ) : max2(DE, F);
        if (TB) {
          const uint32_t X3 = E - D + K7F;   // E > D
          const uint32_t X2 = F - DE + K7F;  // F > max(D, E)
          // bytes: low-half sign of X3, of X2, high-half sign of X3, of X2, each
          // 0x00 or 0xff = 255 x flag; summing Pa x 2^c over the group's
          // registers (one multiply-add each, on the FMA pipe) gives 255 x W
          // mod 2^32, W the plane word with flag c in bit c of each byte
          const uint32_t Pa = perm<0xfbd9>(X3, X2);
          accA = (k & 7) == 0 ? Pa : fmad32(Pa, 1u << (k & 7), accA);
          if (AFFINE) {
            const uint32_t X1 = fadd2(fadd2(Ec[k], K7FME, one), Hol, mone);  // E took the extension
            const uint32_t X0 = fadd2(fadd2(Fup, K7FME, one), Hmup, mone);   // F took the extension
            const uint32_t Pb = perm<0xfbd9>(X1, X0);
            accB = (k & 7) == 0 ? Pb : fmad32(Pb, 1u << (k & 7), accB);
          }
          if ((k & 7) == 7 || k == P - 1) {  // a group of (up to) 8 registers is complete
            // 255 is odd: W = (255 W) x 255^-1 mod 2^32, 255^-1 = 0xfefefeff
            const uint32_t WA = accA * 0xfefefeffu, WB = accB * 0xfefefeffu;
            tbw[k >> 3] = perm<0x5410>(WA, WB);      // low half, group k/8
            tbw[G + (k >> 3)] = perm<0x7632>(WA, WB);  // high half
          }
        }
        const uint32_t Hmn = fadd2(H, MOE, one);
        Hdg = Hc[k];
        Hmup = Hmn;
        Fup = F;
        const uint32_t Hk = EDGE ? (H & KM) : H;  // inactive halves count as 0
        if (LOCAL) {  // two registers fold into the step's max at once
          // 32-bit keys: the half's biased H above a tag 31 - row, so the
          // largest key is the largest H and, among equal H, the smallest i
          const uint32_t key_lo = fmad32(Hk, 65536u, 31u - k);
          const uint32_t key_hi = (Hk & 0xffff0000u) | (31u - (P + k));
          mkey = __vimax3_u32(mkey, key_lo, key_hi);
        }
        if constexpr (EDGE) {
          Hc[k] = select_bits(KM, H, Hc[k]);
          if (AFFINE) Ec[k] = select_bits(KM, E, Ec[k]);
          Hm[k] = select_bits(KM, Hmn, Hm[k]);
        } else {
          Hc[k] = H;
          if (AFFINE) Ec[k] = E;
          Hm[k] = Hmn;
        }
      }
    };
    regs(edge_tag);
    outH = Hc[P - 1];
    outF = Fup;
    Flast = Fup;
    if (TB) {
#pragma unroll
      for (int w = 0; w < WPS; ++w) PP.tb[tb_base + ((int64_t)t * WPS + w) * 32 + lane] = tbw[w];
    }
    if (lane == 31 && actH && s + 1 < nstrips)
      buf[cH] = make_int2((int)(Hc[P - 1] >> 16), (int)(Fup >> 16));
    // best cell (local): a lane takes the step's largest key only if strictly
    // above its best key (equal keys: the same row at a later column, whose
    // smaller j already stands).  Rows past M stay below a valid cell of their
    // lane already seen; lanes wholly past M keep no best.
    if (LOCAL && top <= M && mkey > bestkey) {
      bestkey = mkey;
      const int row = 31 - (int)(mkey & 0xffffu);
      best.v = (int)(mkey >> 16) - B;
      best.i = top + row;
      best.j = row < P ? cL : cH;
    }
  };
#pragma unroll 1
  for (int t = 0; t < min(63, nsteps); ++t) step(t, std::true_type{});
#pragma unroll 1
  for (int t = 63; t < N; ++t) step(t, std::false_type{});
#pragma unroll 1
  for (int t = max(63, N); t < nsteps; ++t) step(t, std::true_type{});
  if (!LOCAL && s == nstrips - 1 && top <= M && M < top + R) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      if (top + k == M) endH = (int)(Hc[k] & 0xffffu) - B;
      if (top + P + k == M) endH = (int)(Hc[k] >> 16) - B;
    }
  }
  __syncwarp();
}

template <int R, bool LOCAL, bool AFFINE, bool TB, bool GR>
__global__ void __launch_bounds__(FULL_WARPS * 32) k_pack(const FullArgs a) {
  constexpr int HS = 32 * R;
  extern __shared__ __align__(16) int8_t smem[];
  if (launch_idle<GR>(a)) return;  // uniform over the block
  const int A = a.sp.alphabet;
  int8_t *s_sub = smem;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < A * A; t += blockDim.x) s_sub[t] = a.sp.subst[t];
  __syncthreads();
  const int gw = blockIdx.x * FULL_WARPS + wib;
  int2 *buf = a.strip_buf + (size_t)gw * a.strip_stride;

  for (;;) {
    uint32_t t0 = 0;
    if (lane == 0) t0 = atomicAdd(a.counter, 1u);
    t0 = __shfl_sync(PFULL, t0, 0);
    if (t0 >= launch_n<GR>(a)) break;
    const uint32_t *order = launch_order<GR>(a);
    const uint32_t p = order ? order[t0] : t0;
    const BatchDev bv = launch_batch<GR>(a);
    PackPair PP;
    PP.M = (int)bv.q_len[p];
    PP.N = (int)bv.r_len[p];
    PP.q = bv.q_seq + bv.q_off[p];
    PP.r = bv.r_seq + bv.r_off[p];
    PP.o = a.sp.o;
    PP.e = a.sp.e;
    PP.A = A;
    PP.B = pack_bias(a.sp.mode, a.sp.o, a.sp.e, a.sp.smin, a.sp.smax, PP.M, PP.N);
    PP.one = (a.sp.alphabet > 0) ? 1u : 0u;  // 1, unknown to the compiler
    PP.s_sub = s_sub;
    PP.prof = smem + 512 + wib * (A * pack_prof_stride(R));
    PP.tb = TB ? a.tb + a.tbl[p].off : nullptr;
    const int M = PP.M, N = PP.N;
    const int nstrips = (M + HS - 1) / HS;
    Best best{0, INT_MAX, INT_MAX};
    int endH = 0;
    int64_t tb_base = 0;
    for (int s = 0; s < nstrips; ++s) {
      pack_strip<R, LOCAL, AFFINE, TB>(PP, s, tb_base, buf, best, endH);
      if (TB) tb_base += pack_strip_tb_words(1, N, R);
    }
    int score = 0, ei = 0, ej = 0, status = FILTR_ST_OK;
    if (LOCAL) {
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const int ov = __shfl_xor_sync(PFULL, best.v, off);
        const int oi = __shfl_xor_sync(PFULL, best.i, off);
        const int oj = __shfl_xor_sync(PFULL, best.j, off);
        best_put(best, ov, oi, oj);
      }
      if (best.v > 0) {
        score = best.v;
        ei = best.i;
        ej = best.j;
      } else {
        status = FILTR_ST_EMPTY;
      }
    } else {
      const int owner = ((M - 1) % HS) / R;
      score = __shfl_sync(PFULL, endH, owner);
      ei = M;
      ej = N;
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
      res.cells = (uint64_t)M * (uint64_t)N;
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

template <int R, bool LOCAL, bool AFFINE, bool TB, bool GR>
cudaError_t launch_pt(const FullArgs &a, int grid, cudaStream_t s) {
  auto k = k_pack<R, LOCAL, AFFINE, TB, GR>;
  const int smem = pack_smem_bytes(R, a.sp.alphabet);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, FULL_WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int R, bool LOCAL, bool AFFINE, bool TB, bool GR>
int occ_pt(int smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_pack<R, LOCAL, AFFINE, TB, GR>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pack<R, LOCAL, AFFINE, TB, GR>,
                                                FULL_WARPS * 32, smem);
  return nb;
}

#define FILTR_PACK_CASES(X) \
  X(false, false, false)    \
  X(false, false, true)     \
  X(false, true, false)     \
  X(false, true, true)      \
  X(true, false, false)     \
  X(true, false, true)      \
  X(true, true, false)      \
  X(true, true, true)

template <int R, bool GR>
cudaError_t dispatch_pr(const FullArgs &a, int grid, cudaStream_t s) {
  const bool L = a.sp.mode == FILTR_LOCAL, AF = a.sp.affine != 0, T = a.sp.traceback != 0;
#define FILTR_CASE(l, af, t) \
  if (L == l && AF == af && T == t) return launch_pt<R, l, af, t, GR>(a, grid, s);
  FILTR_PACK_CASES(FILTR_CASE)
#undef FILTR_CASE
  return cudaErrorInvalidValue;
}

template <int R, bool GR>
int occ_pr(const ScoreParams &sp) {
  const bool L = sp.mode == FILTR_LOCAL, AF = sp.affine != 0, T = sp.traceback != 0;
  const int smem = pack_smem_bytes(R, sp.alphabet);
#define FILTR_CASE(l, af, t) \
  if (L == l && AF == af && T == t) return occ_pt<R, l, af, t, GR>(smem);
  FILTR_PACK_CASES(FILTR_CASE)
#undef FILTR_CASE
  return 0;
}

}  // namespace
}  // namespace filtr
