// k_pack_graph.cu -- the int16x2 tiled kernel's instances for a captured batch
// pipeline (filtr_graph), R = 8, 16, 24, 32 here and 12, 20, 28 in
// k_pack_graph_mid.cu: the same template with its batch, outputs and order
// slice read on the device, kept apart from the batched call's instances,
// which read their by-value arguments and so hold fewer registers.
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_graph_mid(const FullArgs &a, int R, int grid, cudaStream_t s);
int pack_graph_blocks_per_sm_mid(int R, const ScoreParams &sp);

cudaError_t launch_pack_graph(const FullArgs &a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 8: return dispatch_pr<8, true>(a, grid, s);
    case 16: return dispatch_pr<16, true>(a, grid, s);
    case 24: return dispatch_pr<24, true>(a, grid, s);
    case 32: return dispatch_pr<32, true>(a, grid, s);
    default: return launch_pack_graph_mid(a, R, grid, s);
  }
}

int pack_graph_blocks_per_sm(int R, const ScoreParams &sp) {
  switch (R) {
    case 8: return occ_pr<8, true>(sp);
    case 16: return occ_pr<16, true>(sp);
    case 24: return occ_pr<24, true>(sp);
    case 32: return occ_pr<32, true>(sp);
    default: return pack_graph_blocks_per_sm_mid(R, sp);
  }
}

}  // namespace filtr
