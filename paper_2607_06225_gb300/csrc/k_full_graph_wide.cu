// k_full_graph_wide.cu -- the int32 tiled kernel's captured-pipeline
// instances for R = 24 and 32 (see k_full_graph.cu).
#include "k_full_impl.cuh"

namespace filtr {

cudaError_t launch_full_graph_wide(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (R == 24) return dispatch_r<24, true>(a, grid, s);
  if (R == 32) return dispatch_r<32, true>(a, grid, s);
  return cudaErrorInvalidValue;
}

int full_graph_blocks_per_sm_wide(int R, const ScoreParams &sp) {
  const int smem = full_smem_bytes(R, sp.alphabet);
  if (R == 24) return occ_r<24, true>(sp, smem);
  if (R == 32) return occ_r<32, true>(sp, smem);
  return 0;
}

}  // namespace filtr
