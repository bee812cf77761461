// Forward kernels instantiated for Q = 19, f32 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q19_s0(Op op, const LaunchArgs& a) { return launch_typed<19, float>(op, a); }
}  // namespace xlb
