// Plain-old-data structures shared by the host side of the library and its
// kernels.  No CUDA or torch types: this header compiles as C++ on the host.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define XLB_HD __host__ __device__
#else
#define XLB_HD
#endif

namespace xlb {

// Cell types of the mask (Section 3.5); values are the public ABI codes.
// FWALL is a full-way bounce-back wall (the walls of the Section 5 cavity):
// it is streamed like a fluid cell and its collision reverses every
// population, so its slots hold real state, never ghost values.
enum CellType : uint8_t { FLUID = 0, WALL = 1, LID = 2, INLET = 3, OUTLET = 4, EQ = 5, FWALL = 6 };

// Derived per-cell flag byte written by the mask preparation kernel:
// bits 0-2 hold the cell type, bit 3 marks a fluid-like cell whose update
// needs the per-direction boundary rules (a WALL / LID / EQ cell in its
// stencil, or an inlet / outlet / FWALL cell itself).
constexpr uint8_t FLAG_TYPE = 0x07;
constexpr uint8_t FLAG_SLOW = 0x08;

XLB_HD inline bool fluid_like(int t) { return t == FLUID || t == INLET || t == OUTLET; }

// Cells whose slots hold streamed state (fluid-like and FWALL); the others
// (WALL, LID, EQ) hold ghost values.
XLB_HD inline bool holds_state(int t) { return fluid_like(t) || t == FWALL; }

// Everything one stream-collide launch needs besides the two buffers.
struct StepParams {
  int nx, ny, nz;        // lattice extents (nz = 1 for D2Q9)
  long long plane;       // elements between consecutive population planes
  float omega;           // dt / tau (Eq. 3, Eq. 4)
  int has_mask;          // 0: every cell is fluid and every face periodic
  const uint8_t* flags;  // derived flag byte per cell (FLAG_*), or null
  int has_force;         // exact-difference body force on fluid-like cells
  float F[3];
  float lid_term[27];    // 2 w_i rho_w (c_i . u_lid) / cs^2 for a LID source
  float eq_df[27];       // f_i^eq(rho_eq, u_eq) - w_i (equilibrium-BC cells)
  float eq_rho, eq_u[3];
  float inlet_u[3];      // Zou-He inlet velocity
  const float* inlet_field;  // or per-cell inlet velocities (D x N, component-major), or null
  int inlet_regularized;     // INLET rule: 0 Zou-He, 1 regularized
  int inlet_axis, inlet_sign;  // inward normal n = sign e_axis of the INLET boundary
  int* err;              // device error word for kernels with bounded waits
  // Boundary faces: type (0 = none, WALL, LID, EQ or FWALL) of each whole
  // face plane x = 0, x = nx-1, y = 0, y = ny-1, z = 0, z = nz-1 that the
  // mask fills uniformly (where planes meet WALL wins, then FWALL).  Pulls
  // from a WALL / LID / EQ plane apply the rule by coordinates, pulls from an
  // FWALL plane are plain, and cells of an FWALL plane reverse instead of
  // colliding; every other WALL / LID / EQ source uses ghost values.
  int face[6];
  int has_faces;
  // 16-bit bulk passes: the sources on the x-face planes outside the skipped
  // y / z face rows are served by ghost links, not by rules in the pull
  int x_linked;
  // the x = 0 plane is INLET / the x = nx - 1 plane is OUTLET (outside the
  // y / z face planes): the bulk pass applies the inlet rule / the outflow
  // copy in the lanes of those cells, which are not fix-up cells
  int x_inlet;
  int x_outlet;
  // bulk kernels: 1 when launched on a (x-blocks, ny, nz) grid, 0 when the
  // grid is flattened over rows (ny or nz above the grid limit)
  int grid3;
};

// Ghost link entries are int2 {cell, dir | type << 8 | flags << 16}; LINK_BZ
// marks a WALL link with a Bouzidi wall distance (in a parallel float array).
constexpr int LINK_BZ = 1 << 16;

// Device error codes written to StepParams::err.
constexpr int DEVERR_TIMEOUT = 1;

// Deviation storage: populations are stored as f_i - w_i * RHO0.
constexpr float RHO0 = 1.0f;

}  // namespace xlb
