// k_pack.cu -- instances of the int16x2 tiled kernel (k_pack_impl.cuh) for
// R = 8, 16, 24 and 32 rows per lane, and the dispatch over every packed height
// (R = 12, 20, 28 in k_pack_mid.cu, the heights with an odd number of rows per
// half in k_pack_odd.cu; the translation units compile in parallel).
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_graph(const FullArgs &a, int R, int grid, cudaStream_t s);

cudaError_t launch_pack(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (a.sp.use_band) return cudaErrorInvalidValue;  // unbanded pairs only
  if (a.gd) return launch_pack_graph(a, R, grid, s);  // captured pipeline instances
  switch (R) {
    case 8: return dispatch_pr<8, false>(a, grid, s);
    case 16: return dispatch_pr<16, false>(a, grid, s);
    case 24: return dispatch_pr<24, false>(a, grid, s);
    case 32: return dispatch_pr<32, false>(a, grid, s);
    case 12:
    case 20:
    case 28: return launch_pack_mid(a, R, grid, s);
    default: return launch_pack_odd(a, R, grid, s);
  }
}

int pack_max_blocks_per_sm(int R, const ScoreParams &sp) {
  switch (R) {
    case 8: return occ_pr<8, false>(sp);
    case 16: return occ_pr<16, false>(sp);
    case 24: return occ_pr<24, false>(sp);
    case 32: return occ_pr<32, false>(sp);
    case 12:
    case 20:
    case 28: return pack_mid_blocks_per_sm(R, sp);
    default: return pack_odd_blocks_per_sm(R, sp);
  }
}

}  // namespace filtr
