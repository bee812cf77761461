// KBC kernels instantiated for Q = 27, bf16 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q27_s2_kbc(Op op, const LaunchArgs& a) { return launch_typed<27, __nv_bfloat16, COLL_KBC>(op, a); }
}  // namespace xlb
