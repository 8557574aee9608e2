// k_pack_mid.cu -- instances of the int16x2 tiled kernel (k_pack_impl.cuh) for
// R = 12, 20 and 28 rows per lane: strip heights of 384, 640 and 896 rows
// between the multiples of 256, which cut the last strip's padding.
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_mid(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (a.sp.use_band) return cudaErrorInvalidValue;
  switch (R) {
    case 12: return dispatch_pr<12, false>(a, grid, s);
    case 20: return dispatch_pr<20, false>(a, grid, s);
    case 28: return dispatch_pr<28, false>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int pack_mid_blocks_per_sm(int R, const ScoreParams &sp) {
  switch (R) {
    case 12: return occ_pr<12, false>(sp);
    case 20: return occ_pr<20, false>(sp);
    case 28: return occ_pr<28, false>(sp);
    default: return 0;
  }
}

}  // namespace filtr
