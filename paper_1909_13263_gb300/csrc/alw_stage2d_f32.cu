// Persistent 2D stage-kernel instantiations for one float variant, 64 x 32 tiles.
#include "alw_launch2d.cuh"

namespace alw {
int launch_stage2d_f32(const Stage2DParams &prm, void *stream) {
  if (prm.tile_w == kTile2DXNarrow) return launch_stage2d_f32_narrow(prm, stream);
  return launch2d_impl<P_F32, kTile2DX>(prm, stream);
}
int stage2d_grid_cap_f32(int weights, int tile_w) {
  if (tile_w == kTile2DXNarrow) return stage2d_grid_cap_f32_narrow(weights);
  return grid_cap_impl<P_F32, kTile2DX>(weights);
}
}  // namespace alw
