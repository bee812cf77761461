// KBC kernels instantiated for Q = 9, f16 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q9_s1_kbc(Op op, const LaunchArgs& a) { return launch_typed<9, __half, COLL_KBC>(op, a); }
}  // namespace xlb
