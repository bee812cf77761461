// Forward kernels instantiated for Q = 9, f16 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q9_s1(Op op, const LaunchArgs& a) { return launch_typed<9, __half>(op, a); }
}  // namespace xlb
