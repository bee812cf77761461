// Forward kernels instantiated for Q = 19, f16 storage.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q19_s1(Op op, const LaunchArgs& a) { return launch_typed<19, __half>(op, a); }
}  // namespace xlb
