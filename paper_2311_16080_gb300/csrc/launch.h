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
  OP_BOUNDARY = 8,       // ghost values of the boundary links + fix-up cell recompute
  OP_WALL_FORCE = 9,     // block partial sums of the momentum-exchange force:
                         // min(ceil(n_links / 256), partial_capacity) rows, at least 1
  OP_KE_PARTIAL = 10,    // block partial sums of the kinetic energy over a box:
                         // min(ceil(box cells / ROW_BLOCK), partial_capacity) rows, at least 1
  OP_FACE_GHOSTS = 11    // ghost values of the boundary faces from the stored state in dst
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
  const int2* links;           // OP_BOUNDARY / OP_WALL_FORCE ghost links {cell, dir | type << 8 | flags << 16}
  const int2* link_cells;      // OP_BOUNDARY: per link {source cell x - c_i, FLUID cell x + c_i or -1}
  const float* link_q;         // Bouzidi wall distance of each LINK_BZ link (or null)
  long long n_links;
  const int* fix;              // OP_BOUNDARY fix-up cells (INLET, OUTLET, FWALL off the faces)
  long long n_fix;
  int fix_mode;                // OP_BOUNDARY: how the fix-up cells are handled (FixMode)
  void* side;                  // OP_BOUNDARY: Q x n_fix side buffer of the storage type
  int box_lo[3], box_ext[3];   // OP_KE_PARTIAL: first cell and extent of the box per axis
  int vec_width;               // OP_STEP_VEC: cells per thread (2 or 4)
  void* stream;
};

// Fix-up cells in the boundary pass (k_boundary).
enum FixMode { FIX_STORED = 0, FIX_RECOMPUTE = 1, FIX_SIDE_COMMIT = 2, FIX_SIDE_COMPUTE = 3 };

// Returns 0 on a successful launch request, a negative code for an invalid
// combination (the caller then reports XLB_ERR_ARG / XLB_ERR_UNSUPPORTED).
int launch_d2q9(Op op, const LaunchArgs& a);
int launch_d3q19(Op op, const LaunchArgs& a);
int launch_d3q27(Op op, const LaunchArgs& a);

// Number of blocks the row-mapped kernels launch for a lattice (partials).
long long row_blocks(const StepParams& p);

// Mask preparation: validates codes (< 7), writes flag bytes; err_word[0] is
// set to 1 on an invalid code, err_word[2] where an INLET, OUTLET or FWALL
// cell occurs.  Q picks the stencil used for the FLAG_SLOW test.
int launch_mask_prepare(int Q, const uint8_t* mask, uint8_t* flags, int nx, int ny, int nz, int* err_word,
                        void* stream);
// The six boundary planes of a device mask into `out` (compact, plane by
// plane: see the face detection in api.cu).
int launch_extract_planes(const uint8_t* mask, int nx, int ny, int nz, uint8_t* out, void* stream);
// n floats from src to dst by a kernel (src or dst may be mapped host memory).
int launch_copy_f32(const float* src, float* dst, long long n, void* stream);
int launch_reduce_final(const double* partial, long long n, double* out, void* stream);
// FP64 sum of squares of n floats (device memory) into column 0 of
// min(ceil(n / 2048), capacity) partial rows (at least 1); returns the rows used.
long long launch_sum_squares(const float* x, long long n, double* partial, long long capacity, void* stream);

// Boundary tables of a mask by compaction: mode 0 selects the FLUID cells
// (and FWALL cells of FWALL faces) whose source in direction `dir` is WALL /
// LID / EQ (written as links {cell, dir | type << 8}), mode 1 the fix-up
// cells (written to `cells`).  Per block of 256 cells: counts, then ordered writes at the
// exclusive offsets of the counts.
long long bnd_list_blocks(long long n);
// `face` (6 types, or null) lists the described boundary faces: links whose
// source lies on one are left out (the pull applies those rules itself).
// x_in / x_out: the INLET cells of x = 0 / OUTLET cells of x = nx - 1 are
// served by the bulk pass: they are not fix-up cells, and their links are
// listed like those of FLUID cells.
// One launch each evaluates every table: counts / offs are indexed
// [pass * chunks + chunk] (chunks of bnd_list_blocks), pass 1..Q-1 the links
// of direction pass, pass Q the fix-up cells.
int launch_pred_count(int Q, const int* face, bool x_in, bool x_out, const uint8_t* flags, int nx, int ny, int nz,
                      int* counts, void* stream);
int launch_pred_write(int Q, const int* face, bool x_in, bool x_out, const uint8_t* flags, int nx, int ny, int nz,
                      const long long* offs, int2* links, int* cells, void* stream);
// Per link {cell x, dir i | ...}: the source cell x - c_i (periodic) and the
// cell x + c_i when it is FLUID, else -1 (the boundary pass's Bouzidi partner).
int launch_link_cells(int Q, const int2* links, long long n, const uint8_t* flags, int nx, int ny, int nz,
                      int2* cells, void* stream);

}  // namespace xlb
