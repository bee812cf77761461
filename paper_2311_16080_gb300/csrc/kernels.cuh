// Kernel templates of the forward path.  Each fwd_q*_*.cu translation unit
// instantiates them for one lattice and one storage type through
// launch_typed; dispatch.cu routes (Q, storage) to those entry points.
//
// Thread mapping: one thread per cell; a block covers ROW_BLOCK consecutive x
// of one (y, z) row and the grid is flattened over (x-blocks, rows), so every
// warp touches 32 consecutive populations of each plane (coalesced).
#pragma once
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "launch.h"

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
template <int Q, int COLL>
struct MinBlocks {
  static constexpr int value = (COLL == 2) ? 4 : (Q == 27 ? 8 : (Q == 19 ? 9 : 12));
};

// Fused pull-stream + collide (+ body force): one lattice update per cell.
// src holds post-collision populations h_{t-1}; dst receives h_t = C(S_bc(h_{t-1})).
// The periodic pull is issued before the cell's flag byte is known (no
// dependent load in front of the 19/27 population loads); cells whose stencil
// touches a boundary then patch the affected directions.  Solid and EQ cells
// are computed but not stored: no rule ever reads their values.
template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK, MinBlocks<Q, COLL>::value)
    k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int fl = p.has_mask ? __ldg(p.flags + c.self) : 0;
  Nbr nb;
  make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
  float df[Q];
  pull_periodic<Q, S>(src, p.plane, nb, df);
  if (fl & FLAG_SLOW) slow_rules<Q, S>(src, p, c.x, c.y, c.z, c.self, fl & FLAG_TYPE, nb, df);
  collide<Q, COLL>(df, p);
  if (!fluid_like(fl & FLAG_TYPE)) return;
  S* out = dst + c.self;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    Store<S>::st(out, df[i]);
    out += p.plane;
  }
}

// Collision only, in place, on a state that holds post-stream populations
// (used once after initialisation, which stores f_0 rather than h).
template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_collide_local(S* f, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  if (p.has_mask && !fluid_like(p.flags[c.self] & FLAG_TYPE)) return;
  float df[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) df[i] = Store<S>::ld_plain(f + (long long)i * p.plane + c.self);
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
    pull_cell<Q, S>(f, p, c.x, c.y, c.z, c.self, fl, nb, df);
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

template <int Q, typename S>
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
      if (a.coll == COLL_NONE)
        k_stream_collide<Q, S, COLL_NONE><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, p);
      else if (a.coll == COLL_BGK)
        k_stream_collide<Q, S, COLL_BGK><<<grid, block, 0, st>>>((const S*)a.src, (S*)a.dst, p);
      else if (Q != 19)
        k_stream_collide<Q, S, (Q == 19 ? COLL_BGK : COLL_KBC)><<<grid, block, 0, st>>>((const S*)a.src,
                                                                                          (S*)a.dst, p);
      else
        return -2;
      break;
    case OP_COLLIDE_LOCAL:
      if (a.coll == COLL_NONE)
        k_collide_local<Q, S, COLL_NONE><<<grid, block, 0, st>>>((S*)a.dst, p);
      else if (a.coll == COLL_BGK)
        k_collide_local<Q, S, COLL_BGK><<<grid, block, 0, st>>>((S*)a.dst, p);
      else if (Q != 19)
        k_collide_local<Q, S, (Q == 19 ? COLL_BGK : COLL_KBC)><<<grid, block, 0, st>>>((S*)a.dst, p);
      else
        return -2;
      break;
    case OP_INIT:
      k_init<Q, S><<<grid, block, 0, st>>>((S*)a.dst, p, a.rho, a.u, a.ucs);
      break;
    case OP_MACRO:
      k_macroscopic<Q, S><<<grid, block, 0, st>>>((const S*)a.src, p, a.kind_h, a.rho_out, a.u_out, a.ucs);
      break;
    case OP_REDUCE_PARTIAL:
      if (a.partial_capacity < nblk) return -3;
      k_reduce_partial<Q, S><<<grid, block, 0, st>>>((const S*)a.src, p, a.kind_h, a.partial);
      break;
    default:
      return -4;
  }
  return 0;
}

}  // namespace xlb
