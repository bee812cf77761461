// Forward kernels instantiated for Q = 27, f16 storage, NONE and BGK
// collisions, plus the collision-independent kernels.
#include "kernels.cuh"

namespace xlb {
int launch_fwd_q27_s1(Op op, const LaunchArgs& a) {
  if (a.coll == COLL_NONE && (op == OP_STEP || op == OP_STEP_VEC || op == OP_BOUNDARY || op == OP_COLLIDE_LOCAL))
    return launch_typed<27, __half, COLL_NONE>(op, a);
  return launch_typed<27, __half, COLL_BGK>(op, a);
}
}  // namespace xlb
