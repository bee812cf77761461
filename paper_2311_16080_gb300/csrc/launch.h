// Host-side launch interface between the C ABI (api.cu) and the per-lattice
// kernel translation units.  Plain pointers and sizes only.
#pragma once
#include <stdint.h>

#include "xlb_types.h"

namespace xlb {

enum Op {
  OP_STEP = 0,           // fused stream + collide: dst = C(S_bc(src))
  OP_COLLIDE_LOCAL = 1,  // in place on dst: dst = C(dst)
  OP_INIT = 2,           // dst = f^eq(rho, u) (and the boundary cells' values)
  OP_MACRO = 3,          // rho_out, u_out from src
  OP_REDUCE_PARTIAL = 4  // block partial sums of mass and momentum
};

struct LaunchArgs {
  StepParams p;
  int storage;  // 0 f32, 1 f16, 2 bf16
  int coll;     // Collision
  const void* src;
  void* dst;
  const float* rho;  // OP_INIT inputs (may be null)
  const float* u;
  long long ucs;     // component stride of u / u_out (elements)
  int kind_h;        // src holds post-collision populations (pull needed)
  float* rho_out;
  float* u_out;
  double* partial;
  long long partial_capacity;  // rows of 4 doubles available in partial
  void* stream;
};

// Returns 0 on a successful launch request, a negative code for an invalid
// combination (the caller then reports XLB_ERR_ARG / XLB_ERR_UNSUPPORTED).
int launch_d2q9(Op op, const LaunchArgs& a);
int launch_d3q19(Op op, const LaunchArgs& a);
int launch_d3q27(Op op, const LaunchArgs& a);

// Number of blocks the row-mapped kernels launch for a lattice (partials).
long long row_blocks(const StepParams& p);

// Mask preparation: validates codes (< 6), writes flag bytes; err_word is set
// to 1 on an invalid code.  Q picks the stencil used for the FLAG_SLOW test.
int launch_mask_prepare(int Q, const uint8_t* mask, uint8_t* flags, int nx, int ny, int nz, int* err_word,
                        void* stream);
int launch_reduce_final(const double* partial, long long n, double* out, void* stream);

}  // namespace xlb
