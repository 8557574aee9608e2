// k_xdrop16.cu -- the X-drop instances of the packed antidiagonal sweep
// (k_xdrop16_impl.cuh).
#include "k_xdrop16_impl.cuh"

namespace filtr {

cudaError_t launch_xdrop16_x(const FullArgs &a, int W, int grid, uint32_t *overflow,
                             uint32_t *n_overflow, cudaStream_t s) {
  return x16_launch_any<false>(a, W, grid, overflow, n_overflow, X16Knobs{a.x16_rebase}, s);
}

int xdrop16_x_blocks_per_sm(int W, const ScoreParams &sp) { return x16_occ_any<false>(W, sp); }

}  // namespace filtr
