// Reverse-mode kernels instantiated for Q = 19, f16 storage.
#include "adjoint_kernels.cuh"

namespace xlb {
int launch_adj_q19_s1(AdjOp op, const AdjointArgs& a) { return launch_adj_typed<19, __half>(op, a); }
}  // namespace xlb
