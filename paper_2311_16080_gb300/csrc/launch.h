// Host-side launch interface between the C ABI (api.cu) and the per-lattice
// kernel translation units.  Plain pointers and sizes only.
#pragma once
#include <stdint.h>
#include <vector_types.h>

#include "xlb_types.h"

namespace xlb {

enum Op {
  OP_STEP = 0,           // fused stream + collide: dst = C(S_bc(src))
  OP_COLLIDE_LOCAL = 1,  // in place on dst: dst = C(dst)
  OP_INIT = 2,           // dst = f^eq(rho, u) (and the boundary cells' values)
  OP_MACRO = 3,          // rho_out, u_out from src
  OP_REDUCE_PARTIAL = 4, // block partial sums of mass and momentum
  OP_STEP_VEC = 7,       // fused stream + collide, V cells per thread, vector loads
  OP_BOUNDARY = 8        // ghost values of the boundary links + inlet / outlet recompute
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
  const int2* links;           // OP_BOUNDARY ghost links {cell, dir | type << 8}
  long long n_links;
  const int* fix;              // OP_BOUNDARY inlet / outlet cells
  long long n_fix;
  int recompute;               // OP_BOUNDARY: recompute the inlet / outlet cells from src
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

// Boundary tables of a mask: per block of 256 cells the number of links and
// of inlet / outlet cells (counts[2b], counts[2b+1]); then, at the exclusive
// offsets offs[2b], offs[2b+1], the links {cell, dir | type << 8} and the
// inlet / outlet cells, in ascending cell order.
long long bnd_list_blocks(long long n);
int launch_bnd_count(int Q, const uint8_t* flags, int nx, int ny, int nz, int* counts, void* stream);
int launch_bnd_write(int Q, const uint8_t* flags, int nx, int ny, int nz, const long long* offs, int2* links,
                     int* fix, void* stream);

}  // namespace xlb
