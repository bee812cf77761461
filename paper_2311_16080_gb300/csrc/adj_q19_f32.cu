// Reverse-mode kernels instantiated for Q = 19, f32 storage.
#include "adjoint_kernels.cuh"

namespace xlb {
int launch_adj_q19_s0(AdjOp op, const AdjointArgs& a) { return launch_adj_typed<19, float>(op, a); }
}  // namespace xlb
