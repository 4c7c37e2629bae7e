// Persistent 2D stage-kernel instantiations for one float variant, 64 x 32 tiles.
#include "alw_launch2d.cuh"

namespace alw {
int launch_stage2d_mixed(const Stage2DParams &prm, void *stream) {
  if (prm.tile_w == kTile2DXNarrow) return launch_stage2d_mixed_narrow(prm, stream);
  return launch2d_impl<P_MIXED, kTile2DX>(prm, stream);
}
int stage2d_grid_cap_mixed(int weights, int tile_w) {
  if (tile_w == kTile2DXNarrow) return stage2d_grid_cap_mixed_narrow(weights);
  return grid_cap_impl<P_MIXED, kTile2DX>(weights);
}
}  // namespace alw
