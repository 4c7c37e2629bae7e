// Persistent 2D stage-kernel instantiations for one float variant, narrow 32 x 32 tiles (batches).
#include "alw_launch2d.cuh"

namespace alw {
int launch_stage2d_mixed_narrow(const Stage2DParams &prm, void *stream) {
  return launch2d_impl<P_MIXED, kTile2DXNarrow>(prm, stream);
}
int stage2d_grid_cap_mixed_narrow(int weights) { return grid_cap_impl<P_MIXED, kTile2DXNarrow>(weights); }
}  // namespace alw
