// k_pack_graph_mid.cu -- the int16x2 tiled kernel's captured-pipeline
// instances for R = 12, 20 and 28 (see k_pack_graph.cu); the heights with an odd
// number of rows per half are in k_pack_graph_odd.cu.
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_graph_odd(const FullArgs &a, int R, int grid, cudaStream_t s);
int pack_graph_odd_blocks_per_sm(int R, const ScoreParams &sp);

cudaError_t launch_pack_graph_mid(const FullArgs &a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 12: return dispatch_pr<12, true>(a, grid, s);
    case 20: return dispatch_pr<20, true>(a, grid, s);
    case 28: return dispatch_pr<28, true>(a, grid, s);
    default: return launch_pack_graph_odd(a, R, grid, s);
  }
}

int pack_graph_blocks_per_sm_mid(int R, const ScoreParams &sp) {
  switch (R) {
    case 12: return occ_pr<12, true>(sp);
    case 20: return occ_pr<20, true>(sp);
    case 28: return occ_pr<28, true>(sp);
    default: return pack_graph_odd_blocks_per_sm(R, sp);
  }
}

}  // namespace filtr
