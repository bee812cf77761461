// KBC kernels instantiated for Q = 9, f32 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q9_s0_kbc(Op op, const LaunchArgs& a) { return launch_typed<9, float, COLL_KBC>(op, a); }
}  // namespace xlb
