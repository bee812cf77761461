// Host-side launch interface of the reverse-mode kernels (adjoint.cu).
#pragma once
#include "xlb_types.h"

namespace xlb {

enum AdjOp {
  ADJ_SEED = 0,      // abar_out = dL/df_T from (dL/drho, dL/du) and the state h_{T-1}
  ADJ_STEP = 1,      // abar_out = fbar_t from abar_in = fbar_{t+1} and state = h_{t-1}
  ADJ_STEP0 = 2,     // abar_out = fbar_0 from abar_in = fbar_1 and f_0 = f^eq(init fields)
  ADJ_INIT_GRAD = 3  // grad_rho, grad_u = dL/d(rho0, u0) from abar_in = fbar_0
};

struct AdjointArgs {
  StepParams p;
  int Q, storage, coll;
  const void* state;        // population buffer (storage type)
  const float* abar_in;     // Q planes of FP32 adjoint populations
  float* abar_out;
  const float* fields_in;   // rho-like field (seed: dL/drho; step0 / init grad: rho0)
  const float* fields_in2;  // vector field (seed: dL/du; step0 / init grad: u0)
  float* grad_rho;
  float* grad_u;
  long long ucs;            // component stride of vector fields
  // ADJ_SEED with ke = 1: the cotangents are those of the kinetic energy
  // (1/2) rho |u|^2 summed over the box [box_lo, box_hi) (times scale), formed
  // in the kernel: dL/drho = |u|^2 / 2, dL/du = rho u inside the box
  int ke;
  int box_lo[3], box_hi[3];
  float scale;
  void* stream;
};

int launch_adjoint(AdjOp op, const AdjointArgs& a);

}  // namespace xlb
