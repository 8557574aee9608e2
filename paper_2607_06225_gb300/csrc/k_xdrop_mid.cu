// k_xdrop_mid.cu -- the antidiagonal sweep over Table 1's M/I/D recurrence
// (k_xdrop_impl.cuh with the gap-open source moved from H to the diagonal state
// M), with or without an X-drop threshold, in a translation unit of its own.
#include "k_xdrop_impl.cuh"

namespace filtr {

cudaError_t launch_mid_w(const FullArgs &a, int W, int grid, uint32_t *overflow,
                         uint32_t *n_overflow, cudaStream_t s) {
  return launch_any_w<2>(a, W, grid, overflow, n_overflow, s);
}

int mid_blocks_per_sm(int W, const ScoreParams &sp) { return occ_any_w<2>(W, sp); }

}  // namespace filtr
