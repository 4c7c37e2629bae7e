// Persistent 2D stage-kernel instantiations for one float variant, narrow 32 x 32 tiles (batches).
#include "alw_launch2d.cuh"

namespace alw {
int launch_stage2d_f32_narrow(const Stage2DParams &prm, void *stream) {
  return launch2d_impl<P_F32, kTile2DXNarrow>(prm, stream);
}
int stage2d_grid_cap_f32_narrow(int weights) { return grid_cap_impl<P_F32, kTile2DXNarrow>(weights); }
}  // namespace alw
