// k_pack_odd.cu -- instances of the int16x2 tiled kernel (k_pack_impl.cuh) for
// R = 10, 14 and 18 rows per lane (an odd number of rows in each half), and the
// dispatch to R = 22, 26, 30 in k_pack_odd_hi.cu: strip heights between those
// of the other tiles, which leave less padding past the query's last row.
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_odd_hi(const FullArgs &a, int R, int grid, cudaStream_t s);
int pack_odd_hi_blocks_per_sm(int R, const ScoreParams &sp);

cudaError_t launch_pack_odd(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (a.sp.use_band) return cudaErrorInvalidValue;
  switch (R) {
    case 10: return dispatch_pr<10, false>(a, grid, s);
    case 14: return dispatch_pr<14, false>(a, grid, s);
    case 18: return dispatch_pr<18, false>(a, grid, s);
    default: return launch_pack_odd_hi(a, R, grid, s);
  }
}

int pack_odd_blocks_per_sm(int R, const ScoreParams &sp) {
  switch (R) {
    case 10: return occ_pr<10, false>(sp);
    case 14: return occ_pr<14, false>(sp);
    case 18: return occ_pr<18, false>(sp);
    default: return pack_odd_hi_blocks_per_sm(R, sp);
  }
}

}  // namespace filtr
