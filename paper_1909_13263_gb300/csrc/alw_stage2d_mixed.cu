// Persistent 2D stage-kernel instantiations for one float variant.
#include "alw_launch2d.cuh"

namespace alw {
int launch_stage2d_mixed(const Stage2DParams &prm, void *stream) { return launch2d_impl<P_MIXED>(prm, stream); }
}  // namespace alw
