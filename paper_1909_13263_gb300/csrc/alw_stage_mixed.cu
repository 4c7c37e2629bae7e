// Stage-kernel instantiations for one arithmetic variant.
#include "alw_launch.cuh"

namespace alw {
int launch_stage_mixed(const StageParams &p, void *stream) { return launch_stage_impl<P_MIXED>(p, stream); }
}  // namespace alw
