// Reverse-mode kernels instantiated for Q = 19, bf16 storage.
#include "adjoint_kernels.cuh"

namespace xlb {
int launch_adj_q19_s2(AdjOp op, const AdjointArgs& a) { return launch_adj_typed<19, __nv_bfloat16>(op, a); }
}  // namespace xlb
