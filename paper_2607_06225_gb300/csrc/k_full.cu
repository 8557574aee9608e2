// k_full.cu -- narrow row tiles (R = 8, 16) of the batched tiled kernel, the
// dispatcher over every tile height, and the kernel's shared-memory size.
#include "k_full_impl.cuh"

namespace filtr {

cudaError_t launch_full_wide(const FullArgs &a, int R, int grid, cudaStream_t s);
int full_max_blocks_per_sm_wide(int R, const ScoreParams &sp, int alphabet);

int full_smem_bytes(int R, int alphabet) { return 512 + FULL_WARPS * alphabet * 32 * R; }

int full_max_blocks_per_sm(int R, const ScoreParams &sp, int alphabet) {
  const int smem = full_smem_bytes(R, alphabet);
  if (R == 8) return occ_r<8>(sp, smem);
  if (R == 16) return occ_r<16>(sp, smem);
  return full_max_blocks_per_sm_wide(R, sp, alphabet);
}

cudaError_t launch_full(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (R == 8) return dispatch_r<8>(a, grid, s);
  if (R == 16) return dispatch_r<16>(a, grid, s);
  return launch_full_wide(a, R, grid, s);
}

}  // namespace filtr
