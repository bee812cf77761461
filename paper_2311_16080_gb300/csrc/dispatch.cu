// Dispatch from (lattice, storage) to the per-instantiation translation units.
#include "adjoint.h"
#include "launch.h"

namespace xlb {

#define XLB_FWD(Q) \
  int launch_fwd_q##Q##_s0(Op, const LaunchArgs&); \
  int launch_fwd_q##Q##_s1(Op, const LaunchArgs&); \
  int launch_fwd_q##Q##_s2(Op, const LaunchArgs&);
XLB_FWD(9)
XLB_FWD(19)
XLB_FWD(27)
#undef XLB_FWD
#define XLB_FWD_KBC(Q) \
  int launch_fwd_q##Q##_s0_kbc(Op, const LaunchArgs&); \
  int launch_fwd_q##Q##_s1_kbc(Op, const LaunchArgs&); \
  int launch_fwd_q##Q##_s2_kbc(Op, const LaunchArgs&);
XLB_FWD_KBC(9)
XLB_FWD_KBC(27)
#undef XLB_FWD_KBC

// Collision-dependent ops of a KBC ctx go to the KBC units; everything else to
// the NONE / BGK units (which also hold the collision-independent kernels).
static bool kbc_op(Op op, const LaunchArgs& a) {
  return a.coll == 2 && (op == OP_STEP || op == OP_STEP_VEC || op == OP_BOUNDARY || op == OP_COLLIDE_LOCAL);
}

#define XLB_ADJ(Q) \
  int launch_adj_q##Q##_s0(AdjOp, const AdjointArgs&); \
  int launch_adj_q##Q##_s1(AdjOp, const AdjointArgs&);
XLB_ADJ(9)
XLB_ADJ(19)
#undef XLB_ADJ

static int fwd(int Q, Op op, const LaunchArgs& a) {
  const int s = a.storage;
  if (s < 0 || s > 2) return -5;
  if (kbc_op(op, a)) {
    switch (Q) {
      case 9: return s == 0 ? launch_fwd_q9_s0_kbc(op, a) : s == 1 ? launch_fwd_q9_s1_kbc(op, a) : launch_fwd_q9_s2_kbc(op, a);
      case 27:
        return s == 0 ? launch_fwd_q27_s0_kbc(op, a) : s == 1 ? launch_fwd_q27_s1_kbc(op, a) : launch_fwd_q27_s2_kbc(op, a);
    }
    return -2;
  }
  switch (Q) {
    case 9: return s == 0 ? launch_fwd_q9_s0(op, a) : s == 1 ? launch_fwd_q9_s1(op, a) : launch_fwd_q9_s2(op, a);
    case 19: return s == 0 ? launch_fwd_q19_s0(op, a) : s == 1 ? launch_fwd_q19_s1(op, a) : launch_fwd_q19_s2(op, a);
    case 27: return s == 0 ? launch_fwd_q27_s0(op, a) : s == 1 ? launch_fwd_q27_s1(op, a) : launch_fwd_q27_s2(op, a);
  }
  return -6;
}

int launch_d2q9(Op op, const LaunchArgs& a) { return fwd(9, op, a); }
int launch_d3q19(Op op, const LaunchArgs& a) { return fwd(19, op, a); }
int launch_d3q27(Op op, const LaunchArgs& a) { return fwd(27, op, a); }

// The adjoint is provided for D2Q9 and D3Q19 (the differentiable workloads)
// with FP32 and FP16 storage.
int launch_adjoint(AdjOp op, const AdjointArgs& a) {
  const int s = a.storage;
  if (s < 0 || s > 1) return -5;
  if (a.Q == 9) return s == 0 ? launch_adj_q9_s0(op, a) : launch_adj_q9_s1(op, a);
  if (a.Q == 19) return s == 0 ? launch_adj_q19_s0(op, a) : launch_adj_q19_s1(op, a);
  return -6;
}

}  // namespace xlb
