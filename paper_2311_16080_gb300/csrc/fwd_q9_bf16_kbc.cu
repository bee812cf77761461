// KBC kernels instantiated for Q = 9, bf16 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q9_s2_kbc(Op op, const LaunchArgs& a) { return launch_typed<9, __nv_bfloat16, COLL_KBC>(op, a); }
}  // namespace xlb
