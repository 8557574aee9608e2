// k_zdrop.cu -- the Z-drop instances of the antidiagonal sweep (Sec. 9.3's
// condition; k_xdrop_impl.cuh), in a translation unit of their own so that the
// two instance sets compile in parallel.
#include "k_xdrop_impl.cuh"

namespace filtr {

cudaError_t launch_zdrop_w(const FullArgs &a, int W, int grid, uint32_t *overflow,
                           uint32_t *n_overflow, cudaStream_t s) {
  return launch_any_w<1>(a, W, grid, overflow, n_overflow, s);
}

int zdrop_blocks_per_sm(int W, const ScoreParams &sp) { return occ_any_w<1>(W, sp); }

}  // namespace filtr
