// Stage-kernel instantiations for one arithmetic variant.
#include "alw_launch.cuh"

namespace alw {
int launch_stage_f32(const StageParams &p, void *stream) { return launch_stage_impl<P_F32>(p, stream); }
}  // namespace alw
