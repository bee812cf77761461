// KBC kernels instantiated for Q = 27, f32 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q27_s0_kbc(Op op, const LaunchArgs& a) { return launch_typed<27, float, COLL_KBC>(op, a); }
}  // namespace xlb
