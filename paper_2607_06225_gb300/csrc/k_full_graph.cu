// k_full_graph.cu -- the int32 tiled kernel's instances for a captured batch
// pipeline (filtr_graph), R = 8 and 16 here, 24 and 32 in k_full_graph_wide.cu:
// the same template with its batch, outputs and order slice read on the
// device, kept apart from the batched call's instances, which read their
// by-value arguments and so hold fewer registers.
#include "k_full_impl.cuh"

namespace filtr {

cudaError_t launch_full_graph_wide(const FullArgs &a, int R, int grid, cudaStream_t s);
int full_graph_blocks_per_sm_wide(int R, const ScoreParams &sp);

cudaError_t launch_full_graph(const FullArgs &a, int R, int grid, cudaStream_t s) {
  if (R == 8) return dispatch_r<8, true>(a, grid, s);
  if (R == 16) return dispatch_r<16, true>(a, grid, s);
  return launch_full_graph_wide(a, R, grid, s);
}

int full_graph_blocks_per_sm(int R, const ScoreParams &sp) {
  const int smem = full_smem_bytes(R, sp.alphabet);
  if (R == 8) return occ_r<8, true>(sp, smem);
  if (R == 16) return occ_r<16, true>(sp, smem);
  return full_graph_blocks_per_sm_wide(R, sp);
}

}  // namespace filtr
