// k_pack_odd_hi.cu -- instances of the int16x2 tiled kernel (k_pack_impl.cuh)
// for R = 22, 26 and 30 rows per lane (see k_pack_odd.cu).
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_odd_hi(const FullArgs &a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 22: return dispatch_pr<22, false>(a, grid, s);
    case 26: return dispatch_pr<26, false>(a, grid, s);
    case 30: return dispatch_pr<30, false>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int pack_odd_hi_blocks_per_sm(int R, const ScoreParams &sp) {
  switch (R) {
    case 22: return occ_pr<22, false>(sp);
    case 26: return occ_pr<26, false>(sp);
    case 30: return occ_pr<30, false>(sp);
    default: return 0;
  }
}

}  // namespace filtr
