// Persistent 2D stage-kernel instantiations for one float variant.
#include "alw_launch2d.cuh"

namespace alw {
int launch_stage2d_f32(const Stage2DParams &prm, void *stream) { return launch2d_impl<P_F32>(prm, stream); }
int stage2d_grid_cap_f32(int weights) { return grid_cap_impl<P_F32>(weights); }
}  // namespace alw
