// k_xdrop.cu -- the X-drop instances of the antidiagonal sweep (k_xdrop_impl.cuh)
// and the launch entry points, which pick X-drop or Z-drop instances.
#include "k_xdrop_impl.cuh"

namespace filtr {

cudaError_t launch_zdrop_w(const FullArgs &a, int W, int grid, uint32_t *overflow,
                           uint32_t *n_overflow, cudaStream_t s);
int zdrop_blocks_per_sm(int W, const ScoreParams &sp);
cudaError_t launch_mid_w(const FullArgs &a, int W, int grid, uint32_t *overflow,
                         uint32_t *n_overflow, cudaStream_t s);
int mid_blocks_per_sm(int W, const ScoreParams &sp);

cudaError_t launch_xdrop16_x(const FullArgs &a, int W, int grid, uint32_t *overflow,
                             uint32_t *n_overflow, cudaStream_t s);
cudaError_t launch_xdrop16_z(const FullArgs &a, int W, int grid, uint32_t *overflow,
                             uint32_t *n_overflow, cudaStream_t s);
int xdrop16_x_blocks_per_sm(int W, const ScoreParams &sp);
int xdrop16_z_blocks_per_sm(int W, const ScoreParams &sp);

// one-warp groups run four to a block: the int32 sweep at W = 1, the packed
// sweep at W = 1 and W = 2 (16 slots per thread)
int xd_pairs_per_cta(int W, const ScoreParams &sp) { return (W == 1 || (W == 2 && sp.xd16)) ? 4 : 1; }

int xd_max_blocks_per_sm(int W, const ScoreParams &sp) {
  if (sp.xd16) return sp.zdrop ? xdrop16_z_blocks_per_sm(W, sp) : xdrop16_x_blocks_per_sm(W, sp);
  if (sp.mid) return mid_blocks_per_sm(W, sp);
  return sp.zdrop ? zdrop_blocks_per_sm(W, sp) : occ_any_w<0>(W, sp);
}

cudaError_t launch_xdrop(const FullArgs &a, int W, int grid, uint32_t *overflow, uint32_t *n_overflow,
                         cudaStream_t s) {
  if (a.sp.xd16)
    return a.sp.zdrop ? launch_xdrop16_z(a, W, grid, overflow, n_overflow, s)
                      : launch_xdrop16_x(a, W, grid, overflow, n_overflow, s);
  if (a.sp.mid) return launch_mid_w(a, W, grid, overflow, n_overflow, s);
  if (a.sp.zdrop) return launch_zdrop_w(a, W, grid, overflow, n_overflow, s);
  return launch_any_w<0>(a, W, grid, overflow, n_overflow, s);
}

}  // namespace filtr
