// Reverse-mode kernels instantiated for Q = 9, f16 storage.
#include "adjoint_kernels.cuh"

namespace xlb {
int launch_adj_q9_s1(AdjOp op, const AdjointArgs& a) { return launch_adj_typed<9, __half>(op, a); }
}  // namespace xlb
