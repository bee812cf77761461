// Reverse-mode kernels instantiated for Q = 9, f32 storage.
#include "adjoint_kernels.cuh"

namespace xlb {
int launch_adj_q9_s0(AdjOp op, const AdjointArgs& a) { return launch_adj_typed<9, float>(op, a); }
}  // namespace xlb
