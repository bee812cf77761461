// Kernel templates of the forward path.  Each fwd_q*_*.cu translation unit
// instantiates them for one lattice and one storage type through
// launch_typed; dispatch.cu routes (Q, storage) to those entry points.
//
// Thread mapping: one thread per cell; a block covers ROW_BLOCK consecutive x
// of one (y, z) row and the grid is flattened over (x-blocks, rows), so every
// warp touches 32 consecutive populations of each plane (coalesced).
#pragma once
#include <cuda_runtime.h>

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

// Blocks per SM the forward kernels are compiled for (register budget).
#ifndef XLB_MINB_Q19_16
#define XLB_MINB_Q19_16 9
#endif
template <int Q, typename S, int COLL>
struct MinBlocks {
  static constexpr int value =
      (COLL == 2) ? 5 : (Q == 27 ? 8 : (Q == 19 ? (sizeof(S) == 2 ? XLB_MINB_Q19_16 : 9) : 12));
};

// Bulk pass of an update, one thread per cell: pull-stream + collide
// (+ body force) of every cell as if periodic.  src holds post-collision
// populations h_{t-1} with ghost values in the boundary cells, so the pull is
// exact for every fluid cell; dst receives h_t = C(S_bc(h_{t-1})).  Boundary
// cells get values nobody reads until k_boundary rewrites them; inlet /
// outlet cells are recomputed there too.
// FW: the lattice has FWALL face planes (their cells reverse instead of
// colliding, and pulls from them are plain); the FW = false instance carries
// none of that logic.
template <int Q, typename S, int COLL, bool FW>
__global__ void __launch_bounds__(ROW_BLOCK, MinBlocks<Q, S, COLL>::value)
    k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  Nbr nb;
  make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
  float df[Q];
  const bool on_fwall = pull_periodic<Q, S, FW>(src, p, nb, c.self, c.x, c.y, c.z, df);
  if (FW && COLL != COLL_NONE && on_fwall)
    reverse_populations<Q>(df);
  else
    collide<Q, COLL>(df, p);
  S* out = dst + c.self;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    Store<S>::st(out, df[i]);
    out += p.plane;
  }
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
  Store<S>::st(dst + (long long)i * p.plane + (wx + p.nx * (wy + p.ny * wz)), v);
}

// Ghost value of a WALL link with a Bouzidi wall distance q (Bouzidi,
// Firdaouss and Lallemand 2001; the curved-wall rule Section 4.3 names): the
// value FLUID cell x pulls in direction j, with hi = h_opp(j)(x):
//   q <  1/2: 2q hi + (1 - 2q) h_opp(j)(x + c_j)  (hi if x + c_j is not FLUID)
//   q >= 1/2: hi / (2q) + (1 - 1/(2q)) h_j(x)
// The cells read are FLUID cells of dst, which the boundary pass never writes.
template <int Q, typename S>
__device__ __forceinline__ float bouzidi_ghost(const S* __restrict__ dst, const StepParams& p, int x, int j,
                                               float hi, float q) {
  int dx = 0, dy = 0, dz = 0, io = 0;
#pragma unroll
  for (int jj = 1; jj < Q; ++jj)
    if (jj == j) {
      dx = Lattice<Q>::c(jj, 0);
      dy = Lattice<Q>::c(jj, 1);
      dz = Lattice<Q>::c(jj, 2);
      io = opposite<Q>(jj);
    }
  if (q < 0.5f) {
    const int r = x / p.nx;
    int bx = x - r * p.nx + dx, by = r % p.ny + dy, bz = r / p.ny + dz;
    bx = bx < 0 ? p.nx - 1 : (bx >= p.nx ? 0 : bx);
    by = by < 0 ? p.ny - 1 : (by >= p.ny ? 0 : by);
    bz = bz < 0 ? p.nz - 1 : (bz >= p.nz ? 0 : bz);
    const int b = bx + p.nx * (by + p.ny * bz);
    if ((__ldg(p.flags + b) & FLAG_TYPE) != FLUID) return hi;
    return 2.0f * q * hi + (1.0f - 2.0f * q) * Store<S>::ld_plain(dst + (long long)io * p.plane + b);
  }
  const float inv = 0.5f / q;
  return inv * hi + (1.0f - inv) * Store<S>::ld_plain(dst + (long long)j * p.plane + x);
}

// Boundary pass on dst, after a pass that wrote post-collision values there.
// Threads [0, ceil(n_links / 4)) write the ghost values of the links of FLUID
// cells and of cells on FWALL face planes (4 links each; LINK_BZ links take
// the Bouzidi value with link_q[e]); the next n_fix threads handle one INLET,
// OUTLET or other FWALL cell each: with `recompute`, its update from src with
// the full rules (the bulk pass pulled and collided it as if periodic fluid);
// then the ghosts of its own links.  src is read only by the recomputation,
// which needs the ghosts of the previous state, already in src.
constexpr int LINKS_PER_THREAD = 4;

template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_boundary(const S* __restrict__ src, S* __restrict__ dst,
                                                        const StepParams p, const int2* __restrict__ links,
                                                        const float* __restrict__ link_q, int n_links,
                                                        const int* __restrict__ fix, int n_fix, int recompute) {
  // link threads: LINKS_PER_THREAD links each, strided by the link-thread
  // count so that a warp's loads and stores stay on consecutive entries
  const int n_lt = (n_links + LINKS_PER_THREAD - 1) / LINKS_PER_THREAD;
  const int k = blockIdx.x * ROW_BLOCK + threadIdx.x;
  if (k < n_lt) {
    int2 l[LINKS_PER_THREAD];
    float h[LINKS_PER_THREAD];
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m) {
      const int e = k + m * n_lt;
      l[m] = e < n_links ? __ldg(links + e) : make_int2(-1, 0);
    }
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m) {
      h[m] = 0.f;
      if (l[m].x >= 0 && ((l[m].y >> 8) & 0xff) != EQ) {
        int io = 0;
        const int i = l[m].y & 0xff;
#pragma unroll
        for (int j = 1; j < Q; ++j)
          if (j == i) io = opposite<Q>(j);
        h[m] = Store<S>::ld_plain(dst + (long long)io * p.plane + l[m].x);
      }
    }
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m)
      if (l[m].x >= 0 && (l[m].y & LINK_BZ))
        h[m] = bouzidi_ghost<Q, S>(dst, p, l[m].x, l[m].y & 0xff, h[m], __ldg(link_q + k + m * n_lt));
#pragma unroll
    for (int m = 0; m < LINKS_PER_THREAD; ++m) {
      if (l[m].x < 0) continue;
      const int x = l[m].x, r = x / p.nx;
      write_ghost<Q, S>(dst, p, x - r * p.nx, r % p.ny, r / p.ny, l[m].y & 0xff, (l[m].y >> 8) & 0xff, h[m]);
    }
    return;
  }
  const int kf = k - n_lt;
  if (kf >= n_fix) return;
  const int self = __ldg(fix + kf);
  const int x = self % p.nx;
  const int r = self / p.nx;
  const int y = r % p.ny, z = r / p.ny;
  Nbr nb;
  make_nbr(nb, x, y, z, p.nx, p.ny, p.nz);
  float df[Q];
  if (recompute) {
    const int type = __ldg(p.flags + self) & FLAG_TYPE;
    pull_cell<Q, S>(src, p, x, y, z, type, nb, df);
    if (type == FWALL) {
      if (COLL != COLL_NONE) reverse_populations<Q>(df);
    } else {
      collide<Q, COLL>(df, p);
    }
    S* out = dst + self;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      Store<S>::st(out, df[i]);
      out += p.plane;
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = Store<S>::ld_plain(dst + (long long)i * p.plane + self);
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int t = __ldg(p.flags + src_index<Q>(nb, i)) & FLAG_TYPE;
    if (!holds_state(t)) {
      // the stored (rounded) value, as the link threads read it
      S hs;
      Store<S>::st(&hs, df[opposite<Q>(i)]);
      write_ghost<Q, S>(dst, p, x, y, z, i, t, Store<S>::ld_plain(&hs));
    }
  }
}

// ---------------------------------------------------------------------------
// Vectorised direct kernel.  Each thread owns V consecutive cells of one row
// (x0 = V * slot); a warp covers 32 V consecutive cells and never straddles a
// row.  Every direction is one aligned V-wide load of the source row at x0;
// the pull's x shift by c_x = +-1 takes the missing end element from the
// neighbouring lane with a warp shuffle, and only the lane at the warp's (or
// row's) edge loads it from memory, with the periodic wrap.  Like the one-cell
// kernel it is a bulk pass (ghost values make the pull exact).  Stores are
// V-wide.  Needs nx % V == 0.

template <int Q, typename S, int COLL, int V>
struct VecMinBlocks {
  static constexpr int value = (COLL == 2) ? 5 : (Q * V > 64 ? 3 : 4);
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
  const bool last = !active || x0 + V >= nx;  // no active right neighbour lane
  const int xm = x0 == 0 ? nx - 1 : x0 - 1;    // element left of the vector
  const int xp = x0 + V >= nx ? 0 : x0 + V;    // element right of the vector
  int rb[3][3];
  {
    const int ys[3] = {wrap_m(y, ny), y, wrap_p(y, ny)};
    const int zs[3] = {nz > 1 ? wrap_m(z, nz) : 0, z, nz > 1 ? wrap_p(z, nz) : 0};
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) rb[b][c] = nx * (ys[b] + ny * zs[c]);
  }
  // face types of the source coordinates (x0 + k -+ 1, y -+ 1, z -+ 1)
  int tx[V][3], ty[3] = {0, 0, 0}, tz[3] = {0, 0, 0};
  bool near = false;
#pragma unroll
  for (int k = 0; k < V; ++k) tx[k][0] = tx[k][1] = tx[k][2] = 0;
  if (p.has_faces) {
    const int fy0 = face_code(wrap_m(y, ny), ny), fy2 = face_code(wrap_p(y, ny), ny);
    ty[0] = (fy0 & 1 ? p.face[2] : 0) | (fy0 & 2 ? p.face[3] : 0);
    ty[2] = (fy2 & 1 ? p.face[2] : 0) | (fy2 & 2 ? p.face[3] : 0);
    if (nz > 1) {
      const int fz0 = face_code(wrap_m(z, nz), nz), fz2 = face_code(wrap_p(z, nz), nz);
      tz[0] = (fz0 & 1 ? p.face[4] : 0) | (fz0 & 2 ? p.face[5] : 0);
      tz[2] = (fz2 & 1 ? p.face[4] : 0) | (fz2 & 2 ? p.face[5] : 0);
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int x = x0 + k;
      const int fxm = face_code(x == 0 ? nx - 1 : x - 1, nx), fxp = face_code(x == nx - 1 ? 0 : x + 1, nx);
      tx[k][0] = (fxm & 1 ? p.face[0] : 0) | (fxm & 2 ? p.face[1] : 0);
      tx[k][2] = (fxp & 1 ? p.face[0] : 0) | (fxp & 2 ? p.face[1] : 0);
      near |= (tx[k][0] | tx[k][2]) != 0;
    }
    near |= (ty[0] | ty[2] | tz[0] | tz[2]) != 0;
  }
  const int self0 = x0 + nx * row;
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
    if (i > 0 && near) {
      // sources on a boundary face read the own opposite population instead
      // (lanes next to a face only; the loads join the same phase)
      const S* own = src + (long long)opposite<Q>(i) * p.plane + self0;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int t = face_combine<false>(tx[k][1 - cx], ty[1 - Lattice<Q>::c(i, 1)], tz[1 - Lattice<Q>::c(i, 2)]);
        if (t == WALL || t == LID) v[i][k] = Store<S>::ld(own + k);
      }
    }
    base += p.plane;
  }
  if (near) {
#pragma unroll
    for (int i = 1; i < Q; ++i)
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int t = face_combine<false>(tx[k][1 - Lattice<Q>::c(i, 0)], ty[1 - Lattice<Q>::c(i, 1)],
                                          tz[1 - Lattice<Q>::c(i, 2)]);
        if (t == EQ) v[i][k] = p.eq_df[i];
        if (t == LID) v[i][k] += p.lid_term[i];
      }
  }
#pragma unroll
  for (int k = 0; k < V; ++k) {
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = v[i][k];
    collide<Q, COLL>(d, p);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i][k] = d[i];
  }
  if (!active) return;
  S* out = dst + (long long)nx * row + x0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    VecIO<S, V>::st(out, v[i]);
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
#pragma unroll
  for (int i = 0; i < Q; ++i) Store<S>::st(f + (long long)i * p.plane + c.self, df[i]);
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
#pragma unroll
  for (int i = 0; i < Q; ++i) Store<S>::st(f + (long long)i * p.plane + c.self, df[i]);
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

// Observables of the post-stream state (Eqs. 6-7): rho and the reported
// velocity u = (j + F/2) / rho on fluid-like cells; EQ cells report
// (rho_w, u_w); solid cells report zeros.  u is component-major, stride ucs.
template <int Q, typename S>
__global__ void __launch_bounds__(ROW_BLOCK) k_macroscopic(const S* f, const StepParams p, int kind_h,
                                                           float* rho_out, float* u_out, long long ucs) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int fl = p.has_mask ? p.flags[c.self] : 0;
  const int t = fl & FLAG_TYPE;
  float rho = 0.f, u[3] = {0.f, 0.f, 0.f};
  if (fluid_like(t)) {
    float df[Q];
    post_stream<Q, S>(f, p, c, fl, kind_h, df);
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
    u[2] = j[2] / rho;
  } else if (t == EQ) {
    rho = p.eq_rho;
    u[0] = p.eq_u[0];
    u[1] = p.eq_u[1];
    u[2] = p.eq_u[2];
  }
  if (rho_out) rho_out[c.self] = rho;
  if (u_out) {
    u_out[c.self] = u[0];
    u_out[ucs + c.self] = u[1];
    if (Lattice<Q>::D == 3) u_out[2 * ucs + c.self] = u[2];
  }
}

// Block-level FP64 partial sums of (mass, j_x, j_y, j_z) over fluid-like
// cells of the post-stream state; one row of 4 doubles per block.
template <int Q, typename S>
__global__ void __launch_bounds__(ROW_BLOCK) k_reduce_partial(const S* f, const StepParams p, int kind_h,
                                                              double* partial) {
  CellIdx c;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (cell_of_block(p, c)) {
    const int fl = p.has_mask ? p.flags[c.self] : 0;
    if (fluid_like(fl & FLAG_TYPE)) {
      float df[Q];
      post_stream<Q, S>(f, p, c, fl, kind_h, df);
      // FP64 accumulation of the cell's moments (the populations are w_i + df_i)
      double m = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double fi = weight_d<Q>(i) + (double)df[i];
        m += fi;
        jx += Lattice<Q>::c(i, 0) * fi;
        jy += Lattice<Q>::c(i, 1) * fi;
        jz += Lattice<Q>::c(i, 2) * fi;
      }
      acc[0] = m;
      acc[1] = jx;
      acc[2] = jy;
      acc[3] = jz;
    }
  }
  __shared__ double red[ROW_BLOCK / 32][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[w][k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int q = 0; q < ROW_BLOCK / 32; ++q) s += red[q][k];
      partial[4 * (long long)blockIdx.x + k] = s;
    }
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
      if (p.face[0] == FWALL || p.face[1] == FWALL || p.face[2] == FWALL || p.face[3] == FWALL ||
          p.face[4] == FWALL || p.face[5] == FWALL)
        k_stream_collide<Q, S, COLL, true><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, p);
      else
        k_stream_collide<Q, S, COLL, false><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, p);
      return 0;
    case OP_STEP_VEC: {
      // 16-bit storage, BGK / NONE, D2Q9 / D3Q19 only (FP32 is faster with one
      // cell per thread; on D3Q27 the 4 x 27 live values do not pay), V = 4
      constexpr int V = 4;
      if constexpr (sizeof(S) == 2 && Q != 27 && COLL != COLL_KBC) {
        if (p.nx % V != 0) return -7;
        const long long spr = (p.nx / V + 31) / 32 * 32;
        const long long blocks = (spr * p.ny * p.nz + 127) / 128;
        if (blocks > 0x7fffffffLL) return -1;
        k_sc_vec<Q, S, COLL, V><<<(unsigned)blocks, 128, 0, st>>>((const S*)a.src, (S*)a.dst, p);
        return 0;
      }
      return -7;
    }
    case OP_BOUNDARY: {
      const long long tot = (a.n_links + LINKS_PER_THREAD - 1) / LINKS_PER_THREAD + a.n_fix;
      if (tot <= 0) return 0;
      if (tot > 0x7fffffffLL) return -1;
      const unsigned g = (unsigned)((tot + ROW_BLOCK - 1) / ROW_BLOCK);
      k_boundary<Q, S, COLL><<<g, ROW_BLOCK, 0, st>>>((const S*)a.src, (S*)a.dst, p, a.links, a.link_q,
                                                     (int)a.n_links, a.fix, (int)a.n_fix, a.recompute);
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
        k_macroscopic<Q, S><<<grid, block, 0, st>>>((const S*)a.src, p, a.kind_h, a.rho_out, a.u_out, a.ucs);
        return 0;
      case OP_REDUCE_PARTIAL:
        if (a.partial_capacity < nblk) return -3;
        k_reduce_partial<Q, S><<<grid, block, 0, st>>>((const S*)a.src, p, a.kind_h, a.partial);
        return 0;
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
