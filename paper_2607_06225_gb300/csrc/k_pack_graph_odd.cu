// k_pack_graph_odd.cu -- the int16x2 tiled kernel's captured-pipeline
// instances for R = 10, 14, 18, 22, 26 and 30 (see k_pack_graph.cu).
#include "k_pack_impl.cuh"

namespace filtr {

cudaError_t launch_pack_graph_odd(const FullArgs &a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 10: return dispatch_pr<10, true>(a, grid, s);
    case 14: return dispatch_pr<14, true>(a, grid, s);
    case 18: return dispatch_pr<18, true>(a, grid, s);
    case 22: return dispatch_pr<22, true>(a, grid, s);
    case 26: return dispatch_pr<26, true>(a, grid, s);
    case 30: return dispatch_pr<30, true>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int pack_graph_odd_blocks_per_sm(int R, const ScoreParams &sp) {
  switch (R) {
    case 10: return occ_pr<10, true>(sp);
    case 14: return occ_pr<14, true>(sp);
    case 18: return occ_pr<18, true>(sp);
    case 22: return occ_pr<22, true>(sp);
    case 26: return occ_pr<26, true>(sp);
    case 30: return occ_pr<30, true>(sp);
    default: return 0;
  }
}

}  // namespace filtr
