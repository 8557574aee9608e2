// k_full_wide.cu -- wide row tiles (R = 24, 32) of the batched tiled kernel:
// strips of 768 / 1024 query rows, so queries up to 1024 residues need one
// strip with little padding.
#include "k_full_impl.cuh"

namespace filtr {

int full_max_blocks_per_sm_wide(int R, const ScoreParams &sp, int alphabet) {
  const int smem = full_smem_bytes(R, alphabet);
  if (R == 24) return occ_r<24, false>(sp, smem);
  if (R == 32) return occ_r<32, false>(sp, smem);
  return 0;
}

cudaError_t launch_full_wide(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (R == 24) return dispatch_r<24, false>(a, grid, s);
  if (R == 32) return dispatch_r<32, false>(a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace filtr
