// Reverse-mode kernel templates: the hand-written adjoint of one lattice
// Boltzmann step.  Instantiated per lattice and storage by adj_q*_*.cu.
//
// Forward (Eqs. 1-2): h_t = C(f_t), f_{t+1} = S_bc(h_t), loss L(f_T).
// Reverse:  hbar_t = S_bc^T fbar_{t+1},  fbar_t = J_C(f_t)^T hbar_t.
// S_bc^T gathers in the opposite direction: h_i(x) feeds f_i(x + c_i) when
// x + c_i is fluid-like and f_opp(i)(x) when x + c_i is a WALL or LID cell
// (EQ sources carry no dependence).  One adjoint launch per step reads the
// tape state h_{t-1} (pulled, to rebuild f_t), gathers fbar_{t+1} and writes
// fbar_t: 3 Q values per cell, all coalesced.
//
// VJP of BGK with the exact-difference force, in (rho, j) variables:
//   h = (1 - omega) f + omega f^eq(rho, j)  [+ f^eq(rho, j + F) - f^eq(rho, j)]
//   f^eq_i(rho, j) = w_i [rho + 3 c_i.j + 4.5 (c_i.j)^2 / rho - 1.5 |j|^2 / rho]
//   d f^eq_i / d rho = w_i [1 - 4.5 (c_i.u)^2 + 1.5 |u|^2]
//   d f^eq_i / d j_a = w_i [3 c_ia + 9 (c_i.u) c_ia - 3 u_a]
#pragma once
#include <cuda_runtime.h>

#include "adjoint.h"
#include "kernels.cuh"

namespace xlb {

// (rbar, jbar) = J_{f^eq}(rho, j)^T g
template <int Q>
__device__ __forceinline__ void eq_vjp(float rho, const float (&j)[3], const float (&g)[Q], float& rb,
                                       float (&jb)[3]) {
  const float ir = 1.0f / rho;
  float u[3] = {j[0] * ir, j[1] * ir, j[2] * ir};
  if (Lattice<Q>::D == 2) u[2] = 0.f;
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  rb = 0.f;
  float sw = 0.f, a[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float cu = 0.f;
    if (Lattice<Q>::c(i, 0)) cu += Lattice<Q>::c(i, 0) * u[0];
    if (Lattice<Q>::c(i, 1)) cu += Lattice<Q>::c(i, 1) * u[1];
    if (Lattice<Q>::c(i, 2)) cu += Lattice<Q>::c(i, 2) * u[2];
    const float wg = weight<Q>(i) * g[i];
    rb += wg * (1.0f - 4.5f * cu * cu + 1.5f * usq);
    sw += wg;
    const float k = wg * (3.0f + 9.0f * cu);
    if (Lattice<Q>::c(i, 0)) a[0] += Lattice<Q>::c(i, 0) * k;
    if (Lattice<Q>::c(i, 1)) a[1] += Lattice<Q>::c(i, 1) * k;
    if (Lattice<Q>::c(i, 2)) a[2] += Lattice<Q>::c(i, 2) * k;
  }
  jb[0] = a[0] - 3.0f * u[0] * sw;
  jb[1] = a[1] - 3.0f * u[1] * sw;
  jb[2] = a[2] - 3.0f * u[2] * sw;
}

// fbar = J_C(f)^T hbar for the collision of the ctx (NONE or BGK [+ force]).
template <int Q, int COLL>
__device__ __forceinline__ void collide_vjp(const float (&df)[Q], const float (&hb)[Q], const StepParams& p,
                                            float (&fb)[Q]) {
  if (COLL == COLL_NONE) {
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = hb[i];
    return;
  }
  float drho, j[3];
  moments<Q>(df, drho, j);
  const float rho = 1.0f + drho;
  if (Lattice<Q>::D == 2) j[2] = 0.f;
  float rb, jb[3];
  eq_vjp<Q>(rho, j, hb, rb, jb);
  float wr = p.omega;  // weight of d f^eq(rho, j)
  if (p.has_force) {
    wr = p.omega - 1.0f;
    float jF[3] = {j[0] + p.F[0], j[1] + p.F[1], j[2] + p.F[2]};
    if (Lattice<Q>::D == 2) jF[2] = 0.f;
    float rb2, jb2[3];
    eq_vjp<Q>(rho, jF, hb, rb2, jb2);
    rb = wr * rb + rb2;
    jb[0] = wr * jb[0] + jb2[0];
    jb[1] = wr * jb[1] + jb2[1];
    jb[2] = wr * jb[2] + jb2[2];
  } else {
    rb *= wr;
    jb[0] *= wr;
    jb[1] *= wr;
    jb[2] *= wr;
  }
  const float one_m = 1.0f - p.omega;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    float v = one_m * hb[k] + rb;
    if (Lattice<Q>::c(k, 0)) v += Lattice<Q>::c(k, 0) * jb[0];
    if (Lattice<Q>::c(k, 1)) v += Lattice<Q>::c(k, 1) * jb[1];
    if (Lattice<Q>::c(k, 2)) v += Lattice<Q>::c(k, 2) * jb[2];
    fb[k] = v;
  }
}

template <int Q>
__device__ __forceinline__ int dst_index(const Nbr& nb, int i) {
  return nb.xo[1 + Lattice<Q>::c(i, 0)] + nb.rb[1 + Lattice<Q>::c(i, 1)][1 + Lattice<Q>::c(i, 2)];
}

// hbar(x) = (S_bc^T abar)(x) for a fluid-like cell x.
template <int Q>
__device__ __forceinline__ void gather_adjoint(const float* __restrict__ ain, const StepParams& p, const Nbr& nb,
                                               int self, int slow, float (&hb)[Q]) {
  if (!slow) {
#pragma unroll
    for (int i = 0; i < Q; ++i) hb[i] = __ldg(ain + (long long)i * p.plane + dst_index<Q>(nb, i));
    return;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int d = dst_index<Q>(nb, i);
    const int t = p.flags[d] & FLAG_TYPE;
    if (fluid_like(t))
      hb[i] = __ldg(ain + (long long)i * p.plane + d);
    else if (t == WALL || t == LID)
      hb[i] = __ldg(ain + (long long)opposite<Q>(i) * p.plane + self);
    else
      hb[i] = 0.f;
  }
}

template <int Q, typename S>
__device__ __forceinline__ void zero_out(float* aout, const StepParams& p, int self) {
#pragma unroll
  for (int i = 0; i < Q; ++i) aout[(long long)i * p.plane + self] = 0.f;
}

// f_0 of a fluid-like cell exactly as the forward initialisation stored it:
// f^eq(rho0, u0) rounded through the storage type.
template <int Q, typename S>
__device__ __forceinline__ void init_state(const float* rho0, const float* u0, long long ucs, int self,
                                           float (&df)[Q], float& rho, float (&u)[3]) {
  rho = rho0[self];
  u[0] = u0[self];
  u[1] = u0[ucs + self];
  u[2] = Lattice<Q>::D == 3 ? u0[2 * ucs + self] : 0.f;
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float drho = rho - 1.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) df[i] = weight<Q>(i) * (drho + rho * eq_poly<Q>(i, u, usq));
  CellRound<S> rnd;
  rnd.begin((uint32_t)self, df);
#pragma unroll
  for (int i = 0; i < Q; ++i) df[i] = rnd.rounded(i, df[i]);
}

template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_adjoint_step(const S* __restrict__ hprev,
                                                            const float* __restrict__ ain,
                                                            float* __restrict__ aout, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int fl = p.has_mask ? p.flags[c.self] : 0;
  if (!fluid_like(fl & FLAG_TYPE)) {
    zero_out<Q, S>(aout, p, c.self);
    return;
  }
  Nbr nb;
  make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
  float df[Q], hb[Q], fb[Q];
  pull_cell<Q, S>(hprev, p, c.x, c.y, c.z, fl & FLAG_TYPE, nb, df);
  gather_adjoint<Q>(ain, p, nb, c.self, fl & FLAG_SLOW, hb);
  collide_vjp<Q, COLL>(df, hb, p, fb);
#pragma unroll
  for (int i = 0; i < Q; ++i) aout[(long long)i * p.plane + c.self] = fb[i];
}

template <int Q, typename S, int COLL>
__global__ void __launch_bounds__(ROW_BLOCK) k_adjoint_step0(const float* __restrict__ rho0,
                                                             const float* __restrict__ u0, long long ucs,
                                                             const float* __restrict__ ain,
                                                             float* __restrict__ aout, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int fl = p.has_mask ? p.flags[c.self] : 0;
  if (!fluid_like(fl & FLAG_TYPE)) {
    zero_out<Q, S>(aout, p, c.self);
    return;
  }
  Nbr nb;
  make_nbr(nb, c.x, c.y, c.z, p.nx, p.ny, p.nz);
  float df[Q], hb[Q], fb[Q], rho, u[3];
  init_state<Q, S>(rho0, u0, ucs, c.self, df, rho, u);
  gather_adjoint<Q>(ain, p, nb, c.self, fl & FLAG_SLOW, hb);
  collide_vjp<Q, COLL>(df, hb, p, fb);
#pragma unroll
  for (int i = 0; i < Q; ++i) aout[(long long)i * p.plane + c.self] = fb[i];
}

// dL/df_T = rbar + ubar . (c_i - u) / rho for the observables of the readout
// (u is the reported velocity (j + F/2) / rho under a body force).  The
// cotangents rbar, ubar are read from the given fields, or, with KE, are
// those of the kinetic energy over the box [lo, hi): scale * |u|^2 / 2 and
// scale * rho u inside it, zero outside.
template <int Q, typename S, bool KE>
__global__ void __launch_bounds__(ROW_BLOCK) k_adjoint_seed(const S* __restrict__ h, const float* __restrict__ rbar,
                                                            const float* __restrict__ ubar, long long ucs,
                                                            float* __restrict__ aout, const StepParams p, int3 lo,
                                                            int3 hi, float scale) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int fl = p.has_mask ? p.flags[c.self] : 0;
  if (!fluid_like(fl & FLAG_TYPE)) {
    zero_out<Q, S>(aout, p, c.self);
    return;
  }
  float df[Q];
  post_stream<Q, S>(h, p, c, fl, 1, df);
  float drho, j[3];
  moments<Q>(df, drho, j);
  if (p.has_force) {
    j[0] += 0.5f * p.F[0];
    j[1] += 0.5f * p.F[1];
    j[2] += 0.5f * p.F[2];
  }
  const float rho = 1.0f + drho, ir = 1.0f / rho;
  const float u[3] = {j[0] * ir, j[1] * ir, Lattice<Q>::D == 3 ? j[2] * ir : 0.f};
  float rb = 0.f, ub[3] = {0.f, 0.f, 0.f};
  if (KE) {
    if (c.x >= lo.x && c.x < hi.x && c.y >= lo.y && c.y < hi.y && c.z >= lo.z && c.z < hi.z) {
      rb = scale * 0.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      ub[0] = scale * rho * u[0];
      ub[1] = scale * rho * u[1];
      ub[2] = scale * rho * u[2];
    }
  } else {
    rb = rbar ? rbar[c.self] : 0.f;
    if (ubar) {
      ub[0] = ubar[c.self];
      ub[1] = ubar[ucs + c.self];
      if (Lattice<Q>::D == 3) ub[2] = ubar[2 * ucs + c.self];
    }
  }
  const float ubu = ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float cu = 0.f;
    if (Lattice<Q>::c(i, 0)) cu += Lattice<Q>::c(i, 0) * ub[0];
    if (Lattice<Q>::c(i, 1)) cu += Lattice<Q>::c(i, 1) * ub[1];
    if (Lattice<Q>::c(i, 2)) cu += Lattice<Q>::c(i, 2) * ub[2];
    aout[(long long)i * p.plane + c.self] = rb + (cu - ubu) * ir;
  }
}

// dL/drho0 = rbar + jbar . u0, dL/du0 = rho0 jbar with (rbar, jbar) the
// f^eq VJP of fbar_0 at (rho0, j0 = rho0 u0).
template <int Q>
__global__ void __launch_bounds__(ROW_BLOCK) k_adjoint_init_grad(const float* __restrict__ rho0,
                                                                 const float* __restrict__ u0, long long ucs,
                                                                 const float* __restrict__ ain, float* grad_rho,
                                                                 float* grad_u, const StepParams p) {
  CellIdx c;
  if (!cell_of_block(p, c)) return;
  const int fl = p.has_mask ? p.flags[c.self] : 0;
  float gr = 0.f, gu[3] = {0.f, 0.f, 0.f};
  if (fluid_like(fl & FLAG_TYPE)) {
    float fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = ain[(long long)i * p.plane + c.self];
    const float rho = rho0[c.self];
    float u[3] = {u0[c.self], u0[ucs + c.self], Lattice<Q>::D == 3 ? u0[2 * ucs + c.self] : 0.f};
    const float j[3] = {rho * u[0], rho * u[1], rho * u[2]};
    float rb, jb[3];
    eq_vjp<Q>(rho, j, fb, rb, jb);
    gr = rb + jb[0] * u[0] + jb[1] * u[1] + jb[2] * u[2];
    gu[0] = rho * jb[0];
    gu[1] = rho * jb[1];
    gu[2] = rho * jb[2];
  }
  if (grad_rho) grad_rho[c.self] = gr;
  if (grad_u) {
    grad_u[c.self] = gu[0];
    grad_u[ucs + c.self] = gu[1];
    if (Lattice<Q>::D == 3) grad_u[2 * ucs + c.self] = gu[2];
  }
}

template <int Q, typename S>
int launch_adj_typed(AdjOp op, const AdjointArgs& a) {
  const StepParams& p = a.p;
  const long long nblk = row_blocks(p);
  if (nblk <= 0) return 0;
  if (nblk > 0x7fffffffLL) return -1;
  const dim3 grid((unsigned)nblk), block(ROW_BLOCK);
  cudaStream_t st = (cudaStream_t)a.stream;
  switch (op) {
    case ADJ_SEED: {
      const int3 lo = make_int3(a.box_lo[0], a.box_lo[1], a.box_lo[2]);
      const int3 hi = make_int3(a.box_hi[0], a.box_hi[1], a.box_hi[2]);
      if (a.ke)
        k_adjoint_seed<Q, S, true><<<grid, block, 0, st>>>((const S*)a.state, nullptr, nullptr, a.ucs, a.abar_out,
                                                           p, lo, hi, a.scale);
      else
        k_adjoint_seed<Q, S, false><<<grid, block, 0, st>>>((const S*)a.state, a.fields_in, a.fields_in2, a.ucs,
                                                            a.abar_out, p, lo, hi, 1.0f);
      return 0;
    }
    case ADJ_STEP:
      if (a.coll == COLL_NONE)
        k_adjoint_step<Q, S, COLL_NONE><<<grid, block, 0, st>>>((const S*)a.state, a.abar_in, a.abar_out, p);
      else if (a.coll == COLL_BGK)
        k_adjoint_step<Q, S, COLL_BGK><<<grid, block, 0, st>>>((const S*)a.state, a.abar_in, a.abar_out, p);
      else
        return -2;
      return 0;
    case ADJ_STEP0:
      if (a.coll == COLL_NONE)
        k_adjoint_step0<Q, S, COLL_NONE><<<grid, block, 0, st>>>(a.fields_in, a.fields_in2, a.ucs, a.abar_in,
                                                                 a.abar_out, p);
      else if (a.coll == COLL_BGK)
        k_adjoint_step0<Q, S, COLL_BGK><<<grid, block, 0, st>>>(a.fields_in, a.fields_in2, a.ucs, a.abar_in,
                                                                a.abar_out, p);
      else
        return -2;
      return 0;
    case ADJ_INIT_GRAD:
      k_adjoint_init_grad<Q><<<grid, block, 0, st>>>(a.fields_in, a.fields_in2, a.ucs, a.abar_in, a.grad_rho,
                                                     a.grad_u, p);
      return 0;
  }
  return -4;
}

}  // namespace xlb
