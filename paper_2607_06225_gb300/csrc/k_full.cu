// k_full.cu -- narrow row tiles (R = 8, 16) of the batched tiled kernel, the
// dispatcher over every tile height, and the kernel's shared-memory size.
#include "k_full_impl.cuh"

namespace filtr {

cudaError_t launch_full_wide(const FullArgs &a, int R, int grid, cudaStream_t s);
int full_max_blocks_per_sm_wide(int R, const ScoreParams &sp, int alphabet);
cudaError_t launch_full_graph(const FullArgs &a, int R, int grid, cudaStream_t s);

int full_smem_bytes(int R, int alphabet) { return 512 + FULL_WARPS * alphabet * 32 * R; }

int full_max_blocks_per_sm(int R, const ScoreParams &sp, int alphabet) {
  const int smem = full_smem_bytes(R, alphabet);
  if (R == 8) return occ_r<8, false>(sp, smem);
  if (R == 16) return occ_r<16, false>(sp, smem);
  return full_max_blocks_per_sm_wide(R, sp, alphabet);
}

cudaError_t launch_full(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (a.gd) return launch_full_graph(a, R, grid, s);  // captured pipeline instances
  if (R == 8) return dispatch_r<8, false>(a, grid, s);
  if (R == 16) return dispatch_r<16, false>(a, grid, s);
  return launch_full_wide(a, R, grid, s);
}

}  // namespace filtr
