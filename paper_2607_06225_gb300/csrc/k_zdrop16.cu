// k_zdrop16.cu -- the Z-drop instances of the packed antidiagonal sweep
// (k_xdrop16_impl.cuh), in a translation unit of their own so the two sets
// compile in parallel.
#include "k_xdrop16_impl.cuh"

namespace filtr {

cudaError_t launch_xdrop16_z(const FullArgs &a, int W, int grid, uint32_t *overflow,
                             uint32_t *n_overflow, cudaStream_t s) {
  return x16_launch_any<true>(a, W, grid, overflow, n_overflow, X16Knobs{a.x16_rebase}, s);
}

int xdrop16_z_blocks_per_sm(int W, const ScoreParams &sp) { return x16_occ_any<true>(W, sp); }

}  // namespace filtr
