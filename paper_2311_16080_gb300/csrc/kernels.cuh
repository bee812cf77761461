// Kernel templates of the forward path.  Each fwd_q*_*.cu translation unit
// instantiates them for one lattice and one storage type through
// launch_typed; dispatch.cu routes (Q, storage) to those entry points.
//
// Thread mapping: one thread per cell; a block covers ROW_BLOCK consecutive x
// of one (y, z) row and the grid is flattened over (x-blocks, rows), so every
// warp touches 32 consecutive populations of each plane (coalesced).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "launch.h"
#include "lbm_device.cuh"

namespace xlb {

constexpr int ROW_BLOCK = 128;

struct CellIdx {
  int x, y, z;
  int self;
};

__device__ __forceinline__ bool cell_of_block(const StepParams& p, CellIdx& c) {
  const unsigned nxb = (unsigned)(p.nx + ROW_BLOCK - 1) / ROW_BLOCK;
  const unsigned row = blockIdx.x / nxb;
  const unsigned xb = blockIdx.x - row * nxb;
  c.x = (int)(xb * ROW_BLOCK + threadIdx.x);
  if (c.x >= p.nx) return false;
  c.y = (int)(row % (unsigned)p.ny);
  c.z = (int)(row / (unsigned)p.ny);
  c.self = c.x + p.nx * (int)row;
  return true;
}

// Cell of a bulk-kernel thread: on a (x-blocks, ny, nz) grid when p.grid3,
// else on the grid flattened over rows (cell_of_block).
__device__ __forceinline__ bool cell_of_grid(const StepParams& p, CellIdx& c) {
  if (!p.grid3) return cell_of_block(p, c);
  c.x = (int)(blockIdx.x * ROW_BLOCK + threadIdx.x);
  if (c.x >= p.nx) return false;
  c.y = (int)blockIdx.y;
  c.z = (int)blockIdx.z;
  c.self = c.x + p.nx * (c.y + p.ny * c.z);
  return true;
}

// Blocks per SM the forward kernels are compiled for (register budget).
#ifndef XLB_MINB_Q19_16
#define XLB_MINB_Q19_16 9
#endif
#ifndef XLB_MINB_KBC
#define XLB_MINB_KBC 6
#endif
template <int Q, typename S, int COLL>
struct MinBlocks {
  static constexpr int value =
      (COLL == 2) ? XLB_MINB_KBC : (Q == 27 ? 8 : (Q == 19 ? (sizeof(S) == 2 ? XLB_MINB_Q19_16 : 9) : 12));
};

// Face types, per axis, of the coordinates v - 1, v and v + 1 (periodic) of
// a cell, from the types lo and hi of the boundary face planes at 0 and
// n - 1 (0: no face).  Axes of extent 1 carry no faces.
__device__ __forceinline__ void axis_face_types(int v, int n, int lo, int hi, int (&t)[3]) {
  t[0] = (v == 1 ? lo : 0) | (v == 0 ? hi : 0);
  t[1] = (v == 0 ? lo : 0) | (v == n - 1 ? hi : 0);
  t[2] = (v == n - 1 ? lo : 0) | (v == n - 2 ? hi : 0);
}

// Faces around a cell, packed into one word: the per-axis face types (3 bits
// each) of the coordinates v - 1, v, v + 1 on x, y and z, and flags:
//   SKIP:  the cell lies in a y / z face row of a WALL / LID / EQ face and is
//          a boundary cell itself: it holds no state, its slots take the
//          ghost values its neighbours push (where such a face meets an FWALL
//          plane the edge cell is FWALL and holds state; where it meets a
//          WALL plane it is WALL);
//   XN:    some source of the cell lies on an x-face plane;
//   RN:    some source may lie in a skipped row (a y / z coordinate of the
//          cell or its neighbours is on a face plane);
//   FWALL: the cell lies on an FWALL face only (it reverses).
// With these, a direction's source w = x - c_i of rule type t (the combined
// face types of w's coordinates, 0 for fluid or FWALL) is pulled plainly
// when t = 0 or w is skipped (it then holds the pushed ghost value), and by
// the rule by coordinates otherwise (an x-face cell in an ordinary row).
constexpr uint32_t FC_SKIP = 1u << 27, FC_XN = 1u << 28, FC_RN = 1u << 29, FC_FWALL = 1u << 30;

__device__ __forceinline__ int fc_type(uint32_t fc, int axis, int k) { return (int)(fc >> (3 * (3 * axis + k))) & 7; }

template <bool FW>
__device__ __forceinline__ uint32_t face_code(const StepParams& p, int x, int y, int z) {
  if (!p.has_faces) return 0u;
  // a row two or more planes away from the y / z boundary planes (uniform
  // over a warp, which covers one row) can only meet x-faces: their types
  // follow from four compares per lane
  if (y > 1 && y < p.ny - 2 && (p.nz == 1 || (z > 1 && z < p.nz - 2))) {
    const int tm = (x == 1 ? p.face[0] : 0) | (x == 0 ? p.face[1] : 0);           // x - 1
    const int ts = (x == 0 ? p.face[0] : 0) | (x == p.nx - 1 ? p.face[1] : 0);    // x
    const int tp = (x == p.nx - 1 ? p.face[0] : 0) | (x == p.nx - 2 ? p.face[1] : 0);  // x + 1
    uint32_t fc = (uint32_t)tm | (uint32_t)ts << 3 | (uint32_t)tp << 6;
    if (!p.x_linked && (tm | tp) != 0 && (ts == 0 || (FW && ts == FWALL))) fc |= FC_XN;
    if (FW && ts == FWALL) fc |= FC_FWALL;
    return fc;
  }
  int tx[3], ty[3], tz[3];
  axis_face_types(x, p.nx, p.face[0], p.face[1], tx);
  axis_face_types(y, p.ny, p.face[2], p.face[3], ty);
  axis_face_types(z, p.nz, p.face[4], p.face[5], tz);
  uint32_t fc = 0u;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    fc |= (uint32_t)tx[k] << (3 * k) | (uint32_t)ty[k] << (3 * (3 + k)) | (uint32_t)tz[k] << (3 * (6 + k));
  // x-face sources matter to cells that hold state: not to the boundary
  // cells of an x-face plane themselves (FWALL ones do hold state)
  if (!p.x_linked && (tx[0] | tx[2]) != 0 && (tx[1] == 0 || (FW && tx[1] == FWALL))) fc |= FC_XN;
  if ((ty[0] | ty[1] | ty[2] | tz[0] | tz[1] | tz[2]) != 0) fc |= FC_RN;
  const int self = face_combine<FW>(tx[1], ty[1], tz[1]);
  if (self != 0 && face_combine<FW>(0, ty[1], tz[1]) != 0)
    fc |= FC_SKIP;
  else if (FW && self == 0 && (tx[1] == FWALL || ty[1] == FWALL || tz[1] == FWALL))
    fc |= FC_FWALL;
  return fc;
}

// Rule type of direction i's source and whether that source is a skipped
// cell (its slot then holds the pushed ghost value).
template <int Q, bool FW>
__device__ __forceinline__ int source_rule(uint32_t fc, int i, bool& skipped) {
  const int ry = fc_type(fc, 1, 1 - Lattice<Q>::c(i, 1)), rz = fc_type(fc, 2, 1 - Lattice<Q>::c(i, 2));
  const int t = face_combine<FW>(fc_type(fc, 0, 1 - Lattice<Q>::c(i, 0)), ry, rz);
  skipped = t != 0 && face_combine<FW>(0, ry, rz) != 0;
  return t;
}

// Rules by coordinates for the sources on x-face planes in ordinary rows
// (after a plain pull of the cell): WALL: h_opp(i)(x);  LID: h_opp(i)(x) +
// 2 w_i rho_w (c_i . u_w) / cs^2;  EQ: f_i^eq(rho_w, u_w).
template <int Q, typename S, bool FW>
__device__ __forceinline__ void x_face_rules(const S* __restrict__ src, const StepParams& p, int self, uint32_t fc,
                                             float (&df)[Q]) {
  if (!(fc & FC_RN)) {
    // an ordinary row: the source's type is the x-face's alone, one per side
    const int tm = face_combine<FW>(fc_type(fc, 0, 0), 0, 0), tp = face_combine<FW>(fc_type(fc, 0, 2), 0, 0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (Lattice<Q>::c(i, 0) == 0) continue;
      const int t = Lattice<Q>::c(i, 0) > 0 ? tm : tp;
      if (t == 0) continue;
      if (t == EQ)
        df[i] = p.eq_df[i];
      else
        df[i] = Store<S>::ld(src + (long long)opposite<Q>(i) * p.plane + self) + (t == LID ? p.lid_term[i] : 0.f);
    }
    return;
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (Lattice<Q>::c(i, 0) == 0) continue;
    bool skipped;
    const int t = source_rule<Q, FW>(fc, i, skipped);
    if (t == 0 || skipped) continue;
    if (t == EQ)
      df[i] = p.eq_df[i];
    else
      df[i] = Store<S>::ld(src + (long long)opposite<Q>(i) * p.plane + self) + (t == LID ? p.lid_term[i] : 0.f);
  }
}

// Ghost values for the skipped neighbours of a cell x that holds state: for
// each direction i whose source w = x - c_i is skipped, the value the rule
// gives f_i(x) at the next pull goes into w's slot i (WALL: h_opp(i)(x) as
// stored; LID: that + 2 w_i rho_w (c_i . u_w) / cs^2; EQ: f_i^eq(rho_w, u_w)).
// df: the cell's post-collision values, rnd: how they are rounded into
// storage.  (w, i) determines x, so no two cells write the same slot.
template <int Q, typename S, bool FW>
__device__ __forceinline__ void push_ghosts(S* __restrict__ dst, const StepParams& p, int x, int y, int z,
                                            uint32_t fc, const float (&df)[Q], const CellRound<S>& rnd) {
  Nbr nb;
  make_nbr(nb, x, y, z, p.nx, p.ny, p.nz);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    bool skipped;
    const int t = source_rule<Q, FW>(fc, i, skipped);
    if (!skipped) continue;
    const int o = opposite<Q>(i);
    float v = p.eq_df[i];
    if (t != EQ) v = rnd.rounded(o, df[o]) + (t == LID ? p.lid_term[i] : 0.f);
    const long long slot = (long long)i * p.plane + src_index<Q>(nb, i);
    st_ghost<S>(dst + slot, (uint32_t)slot, v);
  }
}

// Plain periodic pull df_i(x) = h_i(x - c_i) of all Q populations, walking
// the planes with one pointer (a 64-bit add per plane; a product i * plane
// per direction costs more instructions).
template <int Q, typename S>
__device__ __forceinline__ void pull_plain(const S* __restrict__ src, const StepParams& p, const Nbr& nb,
                                           float (&df)[Q]) {
  const S* base = src;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    df[i] = Store<S>::ld(base + src_index<Q>(nb, i));
    base += p.plane;
  }
}

template <int Q, typename S>
__device__ __forceinline__ void store_cell(S* __restrict__ dst, const StepParams& p, int self, const CellRound<S>& rnd,
                                           const float (&df)[Q]) {
  S* out = dst + self;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rnd.st(out, i, df[i]);
    out += p.plane;
  }
}

// Which mechanism delivers the rules of the boundary faces to the bulk pass:
// with 16-bit storage the cells of y / z face rows are skipped and take
// ghost values pushed by the rows next to them, and the sources on x-face
// planes are ghost links (p.x_linked) or, with an FWALL x-face, take the
// rules inside the pull (the kernel is bound by instruction issue: whole
// warps skip or push, and at most the lanes at the ends of a row run face
// logic); FP32 applies every face rule by coordinates
// inside the pull (the kernel is bound by memory traffic, and the face logic
// hides under it).  Both give the same pulled values; the readouts, the
// boundary pass and the adjoint apply the face rules by coordinates and never
// read face cells.
template <typename S>
struct GhostFaces {
  static constexpr bool value = sizeof(S) == 2;
};

// Bulk pass of an update, one thread per cell: pull + collide (+ body force)
// + store.  src holds post-collision populations h_{t-1} whose boundary cells
// carry ghost values (the rule's value for the pulling neighbour), so the
// pull is exact for every cell that holds state; dst receives
// h_t = C(S_bc(h_{t-1})).  Faces (whole boundary planes of one type) as
// GhostFaces describes; cells on FWALL face planes reverse instead of
// colliding (FW).  Other boundary cells get values nobody reads until
// k_boundary rewrites them; inlet / outlet cells are recomputed there too.
template <int Q, typename S, int COLL, bool FW, bool IO = false>
__global__ void __launch_bounds__(ROW_BLOCK, MinBlocks<Q, S, COLL>::value)
    k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, const StepParams p) {
  CellIdx c;
  if (!cell_of_grid(p, c)) return;
  float df[Q];
  uint32_t fc = 0u;
  bool fwall = false;
  // IO (a separate instance, so that the other lattices keep their register
  // budget): an OUTLET plane at x = nx - 1 served here copies the pull of
  // x - 1 in the directions c_x = -1, whose sources x - 1 - c_i lie in its
  // own column; an INLET plane at x = 0 takes the inlet rule
  const bool outl = IO && p.x_outlet && c.x == p.nx - 1;
  if constexpr (GhostFaces<S>::value) {
    fc = face_code<FW>(p, c.x, c.y, c.z);
    if (fc & FC_SKIP) return;
    Nbr nb;
    make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
    if (outl) nb.xo[2] = c.x;
    pull_plain<Q, S>(src, p, nb, df);
    if (fc & FC_XN) x_face_rules<Q, S, FW>(src, p, c.self, fc, df);
    fwall = (fc & FC_FWALL) != 0u;
  } else {
    Nbr nb;
    make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
    if (outl) nb.xo[2] = c.x;
    fwall = pull_periodic<Q, S, FW>(src, p, nb, c.self, c.x, c.y, c.z, df, outl);
  }
  if (IO && p.x_inlet && c.x == 0) inlet_rule<Q>(p, c.self, df);
  if (FW && COLL != COLL_NONE && fwall)
    reverse_populations<Q>(df);
  else
    collide<Q, COLL>(df, p);
  CellRound<S> rnd;
  rnd.begin((uint32_t)c.self, df);
  if (GhostFaces<S>::value && (fc & FC_RN)) push_ghosts<Q, S, FW>(dst, p, c.x, c.y, c.z, fc, df, rnd);
  store_cell<Q, S>(dst, p, c.self, rnd, df);
}

// Ghost values of a stored post-collision state (after a local collision or
// a restored state), for storage types that use them: every cell next to a
// skipped face cell pushes them from its stored values.
template <int Q, typename S, bool FW>
__global__ void __launch_bounds__(ROW_BLOCK) k_face_ghosts(S* f, const StepParams p) {
  CellIdx c;
  if (!cell_of_grid(p, c)) return;
  const uint32_t fc = face_code<FW>(p, c.x, c.y, c.z);
  if (!(fc & FC_RN) || (fc & FC_SKIP)) return;
  float hs[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) hs[i] = Store<S>::ld_plain(f + (long long)i * p.plane + c.self);
  CellRound<S> rnd;  // the values are stored ones: rounding them again is exact
  rnd.begin((uint32_t)c.self, hs);
  push_ghosts<Q, S, FW>(f, p, c.x, c.y, c.z, fc, hs, rnd);
}

// Ghost value of the link (cell x, direction i) whose source w = x - c_i has
// type t: what the boundary rule gives f_i(x) at the next update.
//   WALL: h_opp(i)(x);  LID: h_opp(i)(x) + 2 w_i rho_w (c_i . u_w) / cs^2;
//   EQ: f_i^eq(rho_w, u_w).
// (w, i) determines x, so no two links write the same slot.
template <int Q, typename S>
__device__ __forceinline__ void write_ghost(S* __restrict__ dst, const StepParams& p, int x, int y, int z, int i,
                                            int t, float h_opp) {
  int dx = 0, dy = 0, dz = 0;
  float add = 0.f, eqv = 0.f;
#pragma unroll
  for (int j = 1; j < Q; ++j)
    if (j == i) {
      dx = Lattice<Q>::c(j, 0);
      dy = Lattice<Q>::c(j, 1);
      dz = Lattice<Q>::c(j, 2);
      add = p.lid_term[j];
      eqv = p.eq_df[j];
    }
  int wx = x - dx, wy = y - dy, wz = z - dz;
  wx = wx < 0 ? p.nx - 1 : (wx >= p.nx ? 0 : wx);
  wy = wy < 0 ? p.ny - 1 : (wy >= p.ny ? 0 : wy);
  wz = wz < 0 ? p.nz - 1 : (wz >= p.nz ? 0 : wz);
  const float v = t == EQ ? eqv : (t == LID ? h_opp + add : h_opp);
  const long long slot = (long long)i * p.plane + (wx + p.nx * (wy + p.ny * wz));
  st_ghost<S>(dst + slot, (uint32_t)slot, v);
}

// Boundary pass on dst, after a pass that wrote post-collision values there.
// Threads [0, ceil(n_links / 4)) write the ghost values of the links of FLUID
// cells and of cells on FWALL face planes (4 links each; LINK_BZ links take
// the Bouzidi value with link_q[e]); the next n_fix threads handle one INLET,
// OUTLET or other FWALL cell each (the bulk pass pulled and collided it as if
// periodic fluid), by `mode` (FixMode):
//   FIX_RECOMPUTE:    its update from src with the full rules, stored in dst;
//   FIX_SIDE_COMPUTE: the same update stored in the side buffer
//                     side[i * n_fix + k] only (k_fix_recompute; it runs
//                     beside the bulk pass, which it does not depend on);
//   FIX_SIDE_COMMIT:  the values of the side buffer stored in dst;
//   FIX_STORED:       the values already in dst;
// then (all but FIX_SIDE_COMPUTE) the ghosts of its own links.  src is read
// only by the recomputation, which needs the ghosts of the previous state,
// already in src.
constexpr int LINKS_PER_THREAD = 4;

// One fix-up cell kf of the boundary pass, by `mode` (see k_boundary).
template <int Q, typename S, int COLL>
__device__ __forceinline__ void fix_cell(const S* __restrict__ src, S* __restrict__ dst, const StepParams& p,
                                         const int* __restrict__ fix, int n_fix, int mode, S* __restrict__ side,
                                         int kf) {
  const int self = __ldg(fix + kf);
  const int x = self % p.nx;
  const int r = self / p.nx;
  const int y = r % p.ny, z = r / p.ny;
  Nbr nb;
  make_nbr(nb, x, y, z, p.nx, p.ny, p.nz);
  float df[Q];
  if (mode == FIX_RECOMPUTE || mode == FIX_SIDE_COMPUTE) {
    const int type = __ldg(p.flags + self) & FLAG_TYPE;
    pull_cell<Q, S>(src, p, x, y, z, type, nb, df);
    if (type == FWALL) {
      if (COLL != COLL_NONE) reverse_populations<Q>(df);
    } else {
      collide<Q, COLL>(df, p);
    }
    CellRound<S> rnd;
    rnd.begin((uint32_t)self, df);
    if (mode == FIX_SIDE_COMPUTE) {
#pragma unroll
      for (int i = 0; i < Q; ++i) rnd.st(side + (long long)i * n_fix + kf, i, df[i]);
      return;
    }
    S* out = dst + self;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      rnd.st(out, i, df[i]);
      df[i] = rnd.rounded(i, df[i]);  // the stored value, as the link threads read it
      out += p.plane;
    }
  } else if (mode == FIX_SIDE_COMMIT) {
    S* out = dst + self;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const S v = side[(long long)i * n_fix + kf];
      *out = v;
      df[i] = Store<S>::ld_plain(&v);
      out += p.plane;
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = Store<S>::ld_plain(dst + (long long)i * p.plane + self);
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int t = __ldg(p.flags + src_index<Q>(nb, i)) & FLAG_TYPE;
    if (!holds_state(t)) write_ghost<Q, S>(dst, p, x, y, z, i, t, df[opposite<Q>(i)]);
  }
}

// Ghost value of one link from its precomputed cells (k_link_cells): g.x =
// the source cell w = x - c_i, whose slot i takes the value; g.y = the
// Bouzidi partner x + c_i when it is FLUID, else -1.  h = h_opp(i)(x), hb =
// the Bouzidi partner value; both are FLUID cells of dst, which the boundary
// pass never writes.
template <int Q, typename S>
__device__ __forceinline__ void link_ghost(S* __restrict__ dst, const StepParams& p, int2 l, int2 g, float q,
                                           float h, float hb) {
  const int i = l.y & 0xff, t = (l.y >> 8) & 0xff;
  float add = 0.f, eqv = 0.f;
#pragma unroll
  for (int j = 1; j < Q; ++j)
    if (j == i) {
      add = p.lid_term[j];
      eqv = p.eq_df[j];
    }
  float v = h;
  if (l.y & LINK_BZ) {
    // Bouzidi, Firdaouss and Lallemand (2001), the curved-wall rule Section
    // 4.3 names, with hi = h_opp(i)(x):
    //   q <  1/2: 2q hi + (1 - 2q) h_opp(i)(x + c_i)  (hi if x + c_i is not FLUID)
    //   q >= 1/2: hi / (2q) + (1 - 1/(2q)) h_i(x)
    if (q < 0.5f) {
      v = g.y >= 0 ? 2.0f * q * h + (1.0f - 2.0f * q) * hb : h;
    } else {
      const float inv = 0.5f / q;
      v = inv * h + (1.0f - inv) * hb;
    }
  }
  v = t == EQ ? eqv : (t == LID ? v + add : v);
  const long long slot = (long long)i * p.plane + g.x;
  st_ghost<S>(dst + slot, (uint32_t)slot, v);
}

template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_boundary(const S* __restrict__ src, S* __restrict__ dst,
                                                        const StepParams p, const int2* __restrict__ links,
                                                        const int2* __restrict__ link_cells,
                                                        const float* __restrict__ link_q, int n_links,
                                                        const int* __restrict__ fix, int n_fix, int mode,
                                                        S* __restrict__ side) {
  // link threads: LINKS_PER_THREAD links each, strided by the link-thread
  // count so that a warp's loads and stores stay on consecutive entries; all
  // of a link's reads depend only on its table entries (two rounds of loads)
  const int n_lt = (n_links + LINKS_PER_THREAD - 1) / LINKS_PER_THREAD;
  const int k = blockIdx.x * ROW_BLOCK + threadIdx.x;
  if (k < n_lt) {
    int2 l[LINKS_PER_THREAD], g[LINKS_PER_THREAD];
    float q[LINKS_PER_THREAD], h[LINKS_PER_THREAD], hb[LINKS_PER_THREAD];
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m) {
      const int e = k + m * n_lt;
      const bool ok = e < n_links;
      l[m] = ok ? __ldg(links + e) : make_int2(-1, 0);
      g[m] = ok ? __ldg(link_cells + e) : make_int2(0, -1);
      q[m] = ok && link_q ? __ldg(link_q + e) : 1.0f;
    }
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m) {
      h[m] = hb[m] = 0.f;
      if (l[m].x < 0 || ((l[m].y >> 8) & 0xff) == EQ) continue;
      const int i = l[m].y & 0xff;
      int io = 0;
#pragma unroll
      for (int j = 1; j < Q; ++j)
        if (j == i) io = opposite<Q>(j);
      h[m] = Store<S>::ld_plain(dst + (long long)io * p.plane + l[m].x);
      if (l[m].y & LINK_BZ) {
        if (q[m] >= 0.5f)
          hb[m] = Store<S>::ld_plain(dst + (long long)i * p.plane + l[m].x);
        else if (g[m].y >= 0)
          hb[m] = Store<S>::ld_plain(dst + (long long)io * p.plane + g[m].y);
      }
    }
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m)
      if (l[m].x >= 0) link_ghost<Q, S>(dst, p, l[m], g[m], q[m], h[m], hb[m]);
    return;
  }
  const int kf = k - n_lt;
  if (kf < n_fix) fix_cell<Q, S, COLL>(src, dst, p, fix, n_fix, mode, side, kf);
}

// The fix-up cells' recomputation into the side buffer (FIX_SIDE_COMPUTE),
// which runs beside the bulk pass on another stream.
template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_fix_recompute(const S* __restrict__ src, const StepParams p,
                                                             const int* __restrict__ fix, int n_fix,
                                                             S* __restrict__ side) {
  const int kf = blockIdx.x * ROW_BLOCK + threadIdx.x;
  if (kf < n_fix) fix_cell<Q, S, COLL>(src, nullptr, p, fix, n_fix, FIX_SIDE_COMPUTE, side, kf);
}

// ---------------------------------------------------------------------------
// Vectorised bulk kernel.  Each thread owns V consecutive cells of one row
// (x0 = V * slot); a warp covers 32 V consecutive cells and never straddles a
// row.  Every direction is one aligned V-wide load of the source row at x0;
// the pull's x shift by c_x = +-1 takes the missing end element from the
// neighbouring lane with a warp shuffle, and only the lane at the warp's (or
// row's) edge loads it from memory, with the periodic wrap.  Faces as for
// the one-cell kernel with 16-bit storage: the rows of y / z faces are
// skipped (whole warps) and receive ghost values from the rows next to
// them; sources on x-face planes are ghost links (16-bit storage) or take
// the rule in the lanes at the ends of a row.  Stores are V-wide.  Needs
// nx % V == 0; no FWALL faces.

template <int Q, typename S, int COLL, int V>
struct VecMinBlocks {
  static constexpr int value = (COLL == 2) ? 5 : (Q * V > 64 ? 3 : (Q * V > 32 ? 6 : 8));
};

template <int Q, typename S, int COLL, int V>
__global__ void __launch_bounds__(128, VecMinBlocks<Q, S, COLL, V>::value)
    k_sc_vec(const S* __restrict__ src, S* __restrict__ dst, const StepParams p) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int spr = (nx / V + 31) / 32 * 32;  // slots per row, whole warps
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(t / spr);
  if (row >= ny * nz) return;  // whole warps only
  const int slot = (int)(t - (long long)row * spr);
  const int lane = threadIdx.x & 31;
  const bool active = slot * V < nx;
  const int x0 = active ? slot * V : nx - V;
  const int y = row % ny, z = row / ny;
  // face types of the row's coordinates (uniform over the warp); a row on a
  // WALL / LID / EQ face plane holds ghost values only
  int ty[3] = {0, 0, 0}, tz[3] = {0, 0, 0};
  if (p.has_faces) {
    axis_face_types(y, ny, p.face[2], p.face[3], ty);
    axis_face_types(z, nz, p.face[4], p.face[5], tz);
    if (face_combine<false>(0, ty[1], tz[1]) != 0) return;  // the whole warp
  }
  const bool last = !active || x0 + V >= nx;  // no active right neighbour lane
  const int xm = x0 == 0 ? nx - 1 : x0 - 1;    // element left of the vector
  // element right of the vector; an OUTLET plane at x = nx - 1 served here
  // copies the pull of x - 1 in the directions c_x = -1, whose sources lie in
  // its own column
  const int xp = x0 + V >= nx ? (p.x_outlet ? nx - 1 : 0) : x0 + V;
  int rb[3][3];
  {
    const int ys[3] = {wrap_m(y, ny), y, wrap_p(y, ny)};
    const int zs[3] = {nz > 1 ? wrap_m(z, nz) : 0, z, nz > 1 ? wrap_p(z, nz) : 0};
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) rb[b][c] = nx * (ys[b] + ny * zs[c]);
  }
  float v[Q][V];
  const S* base = src;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = Lattice<Q>::c(i, 0);
    const S* r = base + rb[1 - Lattice<Q>::c(i, 1)][1 - Lattice<Q>::c(i, 2)];
    float w[V];
    VecIO<S, V>::ld(r + x0, w);
    if (cx == 0) {
#pragma unroll
      for (int k = 0; k < V; ++k) v[i][k] = w[k];
    } else if (cx == 1) {  // pull from x - 1
      const float up = __shfl_up_sync(0xffffffffu, w[V - 1], 1);
      v[i][0] = lane > 0 ? up : Store<S>::ld(r + xm);
#pragma unroll
      for (int k = 1; k < V; ++k) v[i][k] = w[k - 1];
    } else {  // pull from x + 1
      const float dn = __shfl_down_sync(0xffffffffu, w[0], 1);
      v[i][V - 1] = (lane < 31 && !last) ? dn : Store<S>::ld(r + xp);
#pragma unroll
      for (int k = 0; k < V - 1; ++k) v[i][k] = w[k + 1];
    }
    base += p.plane;
  }
  const int self0 = x0 + nx * row;
  // an INLET plane at x = 0 served here
  if (p.x_inlet && active && x0 == 0) {
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = v[i][0];
    inlet_rule<Q>(p, self0, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i][0] = d[i];
  }
  // sources on x-face planes (only the lanes at the ends of a row have them;
  // none when ghost links serve them)
  if (p.has_faces && !p.x_linked && (x0 <= 1 || x0 + V >= nx - 1)) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      int tx[3];
      axis_face_types(x0 + k, nx, p.face[0], p.face[1], tx);
      if ((tx[0] | tx[2]) == 0 || tx[1] != 0) continue;  // no x-face source, or an x-face cell itself
      uint32_t fc = (ty[0] | ty[1] | ty[2] | tz[0] | tz[1] | tz[2]) != 0 ? FC_RN : 0u;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        fc |= (uint32_t)tx[a] << (3 * a) | (uint32_t)ty[a] << (3 * (3 + a)) | (uint32_t)tz[a] << (3 * (6 + a));
      float d[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = v[i][k];
      x_face_rules<Q, S, false>(src, p, self0 + k, fc, d);
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i][k] = d[i];
    }
  }
  CellRound<S> rnd[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = v[i][k];
    collide<Q, COLL>(d, p);
    rnd[k].begin((uint32_t)(self0 + k), d);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i][k] = d[i];
  }
  if (!active) return;
  // ghost values for the skipped face rows next to this row (from registers,
  // every lane of the row)
  if (p.has_faces && (ty[0] | ty[2] | tz[0] | tz[2]) != 0) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      int tx[3];
      axis_face_types(x0 + k, nx, p.face[0], p.face[1], tx);
      uint32_t fc = FC_RN;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        fc |= (uint32_t)tx[a] << (3 * a) | (uint32_t)ty[a] << (3 * (3 + a)) | (uint32_t)tz[a] << (3 * (6 + a));
      float d[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = v[i][k];
      push_ghosts<Q, S, false>(dst, p, x0 + k, y, z, fc, d, rnd[k]);
    }
  }
  S* out = dst + (long long)nx * row + x0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
      uint16_t b[V];
#pragma unroll
      for (int k = 0; k < V; ++k) b[k] = rnd[k].bits(i, v[i][k]);
      VecIO<S, V>::st_bits(out, b);
    } else {
      VecIO<S, V>::st(out, v[i]);
    }
    out += p.plane;
  }
}

// Collision only, in place, on a state that holds post-stream populations
// (used once after initialisation, which stores f_0 rather than h).
template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_collide_local(S* f, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int t = p.has_mask ? (p.flags[c.self] & FLAG_TYPE) : FLUID;
  if (!holds_state(t) || (t == FWALL && COLL == COLL_NONE)) return;
  float df[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) df[i] = Store<S>::ld_plain(f + (long long)i * p.plane + c.self);
  if (t == FWALL)
    reverse_populations<Q>(df);
  else
    collide<Q, COLL>(df, p);
  CellRound<S> rnd;
  rnd.begin((uint32_t)c.self, df);
#pragma unroll
  for (int i = 0; i < Q; ++i) rnd.st(f + (long long)i * p.plane + c.self, i, df[i]);
}

// f_0 = f^eq(rho, u) on fluid-like cells (Eq. 5); EQ cells take
// f^eq(rho_w, u_w); solid cells the rest state.  rho / u may be null
// (rho = 1, u = 0); u is component-major with stride ucs.
template <int Q, typename S>
__global__ void __launch_bounds__(ROW_BLOCK) k_init(S* f, const StepParams p, const float* rho_in,
                                                    const float* u_in, long long ucs) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int t = p.has_mask ? (p.flags[c.self] & FLAG_TYPE) : FLUID;
  float df[Q];
  if (fluid_like(t)) {
    const float rho = rho_in ? rho_in[c.self] : 1.0f;
    float u[3] = {0.f, 0.f, 0.f};
    if (u_in) {
      u[0] = u_in[c.self];
      u[1] = u_in[ucs + c.self];
      if (Lattice<Q>::D == 3) u[2] = u_in[2 * ucs + c.self];
    }
    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float drho = rho - 1.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = weight<Q>(i) * (drho + rho * eq_poly<Q>(i, u, usq));
  } else if (t == EQ) {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = p.eq_df[i];
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = 0.f;
  }
  CellRound<S> rnd;
  rnd.begin((uint32_t)c.self, df);
#pragma unroll
  for (int i = 0; i < Q; ++i) rnd.st(f + (long long)i * p.plane + c.self, i, df[i]);
}

// Post-stream populations of a cell: pulled from h (state holds h) or read
// in place (state holds f).
template <int Q, typename S>
__device__ __forceinline__ void post_stream(const S* f, const StepParams& p, const CellIdx& c, int fl, int kind_h,
                                            float (&df)[Q]) {
  if (kind_h) {
    Nbr nb;
    make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
    pull_cell<Q, S>(f, p, c.x, c.y, c.z, fl & FLAG_TYPE, nb, df);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = Store<S>::ld(f + (long long)i * p.plane + c.self);
  }
}

// Readouts of the post-stream state, one kernel for the three of them (so
// that the boundary-aware pull is compiled once per lattice and storage):
//  RD_MACRO:   observables (Eqs. 6-7): rho and the reported velocity
//              u = (j + F/2) / rho on fluid-like cells; EQ cells report
//              (rho_w, u_w); solid cells zeros.  u is component-major, stride ucs.
//  RD_MOMENTS: FP64 block partial sums of (mass, j_x, j_y, j_z) over the
//              fluid-like cells (populations w_i + df_i, bare momentum).
//  RD_KE:      FP64 block partial sums of the kinetic energy (1/2) rho |u|^2
//              of the observables RD_MACRO reports (rho, u formed in FP32, the
//              square and the sum in FP64): the loss of the gradient
//              workloads (Section 6 takes gradients of rollout losses).
// Grid-stride over the cells of the box [lo, lo + ext); one partial row
// (4 doubles) per block for the sums.
enum ReadoutMode { RD_MACRO = 0, RD_MOMENTS = 1, RD_KE = 2 };

template <int Q, typename S>
__global__ void __launch_bounds__(ROW_BLOCK) k_readout(const S* f, const StepParams p, int kind_h, int mode,
                                                       int3 lo, int3 ext, float* rho_out, float* u_out,
                                                       long long ucs, double* partial) {
  const long long nbox = (long long)ext.x * ext.y * ext.z;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long k = blockIdx.x * (long long)ROW_BLOCK + threadIdx.x; k < nbox;
       k += (long long)gridDim.x * ROW_BLOCK) {
    CellIdx c;
    const long long r = k / ext.x;
    c.x = lo.x + (int)(k - r * ext.x);
    c.y = lo.y + (int)(r % ext.y);
    c.z = lo.z + (int)(r / ext.y);
    c.self = c.x + p.nx * (c.y + p.ny * c.z);
    const int fl = p.has_mask ? p.flags[c.self] : 0;
    const int t = fl & FLAG_TYPE;
    float rho = 0.f, u[3] = {0.f, 0.f, 0.f};
    if (fluid_like(t)) {
      float df[Q];
      post_stream<Q, S>(f, p, c, fl, kind_h, df);
      if (mode == RD_MOMENTS) {
        double m = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const double fi = weight_d<Q>(i) + (double)df[i];
          m += fi;
          jx += Lattice<Q>::c(i, 0) * fi;
          jy += Lattice<Q>::c(i, 1) * fi;
          jz += Lattice<Q>::c(i, 2) * fi;
        }
        acc[0] += m;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
        continue;
      }
      float drho, j[3];
      moments<Q>(df, drho, j);
      if (p.has_force) {
        j[0] += 0.5f * p.F[0];
        j[1] += 0.5f * p.F[1];
        j[2] += 0.5f * p.F[2];
      }
      rho = 1.0f + drho;
      u[0] = j[0] / rho;
      u[1] = j[1] / rho;
      u[2] = Lattice<Q>::D == 3 ? j[2] / rho : 0.f;
    } else if (t == EQ) {
      rho = p.eq_rho;
      u[0] = p.eq_u[0];
      u[1] = p.eq_u[1];
      u[2] = Lattice<Q>::D == 3 ? p.eq_u[2] : 0.f;
    }
    if (mode == RD_KE) {
      const double u0 = u[0], u1 = u[1], u2 = u[2];
      acc[0] += 0.5 * (double)rho * (u0 * u0 + u1 * u1 + u2 * u2);
    } else if (mode == RD_MACRO) {
      if (rho_out) rho_out[c.self] = rho;
      if (u_out) {
        u_out[c.self] = u[0];
        u_out[ucs + c.self] = u[1];
        if (Lattice<Q>::D == 3) u_out[2 * ucs + c.self] = u[2];
      }
    }
  }
  if (mode == RD_MACRO) return;
  __shared__ double red[ROW_BLOCK / 32][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_down_sync(0xffffffffu, acc[m], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int m = 0; m < 4; ++m) red[threadIdx.x >> 5][m] = acc[m];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int m = 0; m < 4; ++m) {
      double s = 0.0;
      for (int q = 0; q < ROW_BLOCK / 32; ++q) s += red[q][m];
      partial[4 * (long long)blockIdx.x + m] = s;
    }
}

// ---------------------------------------------------------------------------
// Dispatch: one function per lattice, switching on storage and collision.

// Momentum-exchange force on the WALL cells of the ghost links (Mei et al.
// 2002 in the form of Caiazzo and Junk 2008, the method Section 4.3 names)
// of the update that led to the stored state: f holds h_{t-1} and, in the
// WALL slots, the ghost values f_j(x, t) pulled at step t.  Each link (FLUID
// cell x, pulled direction j, WALL source w = x - c_j) hands the wall
//   c_opp(j) [h_opp(j)(x, t-1) + f_j(x, t)] = -c_j [h_opp(j)(x) + ghost_j(w)],
// populations taken absolute (stored deviation + w_j on each side).  Grid-
// stride over the links; one row (F_x, F_y, F_z, 0) of FP64 sums per block.
template <int Q, typename S>
__global__ void __launch_bounds__(256) k_wall_force(const S* __restrict__ f, const StepParams p,
                                                    const int2* __restrict__ links, long long n_links,
                                                    double* partial) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n_links; e += (long long)gridDim.x * 256) {
    const int2 l = __ldg(links + e);
    if (((l.y >> 8) & 0xff) != WALL) continue;
    const int j = l.y & 0xff;
    int dx = 0, dy = 0, dz = 0, io = 0;
    double wj = 0.0;
#pragma unroll
    for (int jj = 1; jj < Q; ++jj)
      if (jj == j) {
        dx = Lattice<Q>::c(jj, 0);
        dy = Lattice<Q>::c(jj, 1);
        dz = Lattice<Q>::c(jj, 2);
        io = opposite<Q>(jj);
        wj = weight_d<Q>(jj);
      }
    const int x = l.x, r = x / p.nx;
    int wx = x - r * p.nx - dx, wy = r % p.ny - dy, wz = r / p.ny - dz;
    wx = wx < 0 ? p.nx - 1 : (wx >= p.nx ? 0 : wx);
    wy = wy < 0 ? p.ny - 1 : (wy >= p.ny ? 0 : wy);
    wz = wz < 0 ? p.nz - 1 : (wz >= p.nz ? 0 : wz);
    const long long w = wx + (long long)p.nx * (wy + (long long)p.ny * wz);
    const double v = 2.0 * wj + (double)Store<S>::ld_plain(f + (long long)io * p.plane + x) +
                     (double)Store<S>::ld_plain(f + (long long)j * p.plane + w);
    acc[0] -= dx * v;
    acc[1] -= dy * v;
    acc[2] -= dz * v;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  __shared__ double red[256 / 32][3];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) red[threadIdx.x >> 5][k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int q = 0; q < 256 / 32; ++q) s += red[q][k];
      partial[4 * (long long)blockIdx.x + k] = s;
    }
    partial[4 * (long long)blockIdx.x + 3] = 0.0;
  }
}

// Launches the collision-dependent kernels for collision COLL and, for
// COLL == COLL_BGK, also the collision-independent ones (init, readouts).
// One translation unit instantiates this per (Q, storage, collision), so the
// heavy KBC kernels compile in parallel with the rest.
template <int Q, typename S, int COLL>
int launch_typed(Op op, const LaunchArgs& a) {
  const StepParams& p = a.p;
  const long long rows = (long long)p.ny * p.nz;
  const long long nxb = (p.nx + ROW_BLOCK - 1) / ROW_BLOCK;
  const long long nblk = rows * nxb;
  if (nblk <= 0) return 0;
  if (nblk > 0x7fffffffLL) return -1;
  const dim3 grid((unsigned)nblk), block(ROW_BLOCK);
  cudaStream_t st = (cudaStream_t)a.stream;
  switch (op) {
    case OP_STEP:
    case OP_FACE_GHOSTS: {
      // bulk kernels run on an (x-blocks, ny, nz) grid where it fits
      StepParams q = p;
      dim3 g3 = grid;
      if (p.ny <= 65535 && p.nz <= 65535) {
        q.grid3 = 1;
        g3 = dim3((unsigned)nxb, (unsigned)p.ny, (unsigned)p.nz);
      }
      const bool fw = p.face[0] == FWALL || p.face[1] == FWALL || p.face[2] == FWALL || p.face[3] == FWALL ||
                      p.face[4] == FWALL || p.face[5] == FWALL;
      if (op == OP_FACE_GHOSTS) {
        if (!p.has_faces || !GhostFaces<S>::value) return 0;
        if (fw)
          k_face_ghosts<Q, S, true><<<g3, block, 0, st>>>((S*)a.dst, q);
        else
          k_face_ghosts<Q, S, false><<<g3, block, 0, st>>>((S*)a.dst, q);
        return 0;
      }
      if (fw)
        k_stream_collide<Q, S, COLL, true><<<g3, block, 0, st>>>((const S*)a.src, (S*)a.dst, q);
      else if (p.x_inlet || p.x_outlet)
        k_stream_collide<Q, S, COLL, false, true><<<g3, block, 0, st>>>((const S*)a.src, (S*)a.dst, q);
      else
        k_stream_collide<Q, S, COLL, false><<<g3, block, 0, st>>>((const S*)a.src, (S*)a.dst, q);
      return 0;
    }
    case OP_STEP_VEC: {
      // 16-bit storage, BGK, D2Q9 / D3Q19 only (FP32 is faster with one cell
      // per thread; on D3Q27 the V x 27 live values do not pay); V = 4
      // (8-byte words) or 2 (4-byte words)
      if constexpr (sizeof(S) == 2 && Q != 27 && COLL == COLL_BGK) {
        const int V = a.vec_width == 2 ? 2 : 4;
        if (p.nx % V != 0) return -7;
        const long long spr = (p.nx / V + 31) / 32 * 32;
        const long long blocks = (spr * p.ny * p.nz + 127) / 128;
        if (blocks > 0x7fffffffLL) return -1;
        if (V == 2)
          k_sc_vec<Q, S, COLL, 2><<<(unsigned)blocks, 128, 0, st>>>((const S*)a.src, (S*)a.dst, p);
        else
          k_sc_vec<Q, S, COLL, 4><<<(unsigned)blocks, 128, 0, st>>>((const S*)a.src, (S*)a.dst, p);
        return 0;
      }
      return -7;
    }
    case OP_BOUNDARY: {
      const long long tot = (a.n_links + LINKS_PER_THREAD - 1) / LINKS_PER_THREAD + a.n_fix;
      if (tot <= 0) return 0;
      if (tot > 0x7fffffffLL) return -1;
      const unsigned g = (unsigned)((tot + ROW_BLOCK - 1) / ROW_BLOCK);
      if (a.fix_mode == FIX_SIDE_COMPUTE) {
        if (a.n_fix <= 0) return 0;
        k_fix_recompute<Q, S, COLL><<<(unsigned)((a.n_fix + ROW_BLOCK - 1) / ROW_BLOCK), ROW_BLOCK, 0, st>>>(
            (const S*)a.src, p, a.fix, (int)a.n_fix, (S*)a.side);
        return 0;
      }
      k_boundary<Q, S, COLL><<<g, ROW_BLOCK, 0, st>>>((const S*)a.src, (S*)a.dst, p, a.links, a.link_cells,
                                                     a.link_q, (int)a.n_links, a.fix, (int)a.n_fix, a.fix_mode,
                                                     (S*)a.side);
      return 0;
    }
    case OP_COLLIDE_LOCAL:
      k_collide_local<Q, S, COLL><<<grid, block, 0, st>>>((S*)a.dst, p);
      return 0;
    default:
      break;
  }
  if constexpr (COLL == COLL_BGK) {
    switch (op) {
      case OP_INIT:
        k_init<Q, S><<<grid, block, 0, st>>>((S*)a.dst, p, a.rho, a.u, a.ucs);
        return 0;
      case OP_MACRO:
      case OP_REDUCE_PARTIAL:
      case OP_KE_PARTIAL: {
        // readouts over a box: the whole lattice, or the KE box; the sums take
        // min(ceil(box cells / ROW_BLOCK), partial_capacity) blocks, at least 1
        const bool box = op == OP_KE_PARTIAL;
        const int3 lo = box ? make_int3(a.box_lo[0], a.box_lo[1], a.box_lo[2]) : make_int3(0, 0, 0);
        const int3 ext = box ? make_int3(a.box_ext[0], a.box_ext[1], a.box_ext[2]) : make_int3(p.nx, p.ny, p.nz);
        const long long nbox = (long long)ext.x * ext.y * ext.z;
        long long b = (nbox + ROW_BLOCK - 1) / ROW_BLOCK;
        if (op != OP_MACRO && b > a.partial_capacity) b = a.partial_capacity;
        if (b > 0x7fffffffLL) b = 0x7fffffffLL;
        if (b < 1) b = 1;
        const int mode = op == OP_MACRO ? RD_MACRO : (op == OP_REDUCE_PARTIAL ? RD_MOMENTS : RD_KE);
        k_readout<Q, S><<<(unsigned)b, ROW_BLOCK, 0, st>>>((const S*)a.src, p, a.kind_h, mode, lo, ext, a.rho_out,
                                                          a.u_out, a.ucs, a.partial);
        return 0;
      }
      case OP_WALL_FORCE: {
        // blocks: one per 256 links, at most the rows the partial buffer holds
        long long b = (a.n_links + 255) / 256;
        if (b > a.partial_capacity) b = a.partial_capacity;
        if (b < 1) b = 1;
        k_wall_force<Q, S><<<(unsigned)b, 256, 0, st>>>((const S*)a.src, p, a.links, a.n_links, a.partial);
        return 0;
      }
      default:
        break;
    }
  }
  return -4;
}

}  // namespace xlb
