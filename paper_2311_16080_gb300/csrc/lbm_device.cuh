// Device functions of the fused stream-collide update: neighbour addressing,
// the pull stream with the mask's boundary rules, moments, equilibrium, BGK
// and KBC collisions and the exact-difference body force.
//
// All arithmetic is FP32 on deviations df_i = f_i - w_i (rho0 = 1):
//   rho = 1 + sum_i df_i                       (Eq. 6)
//   j   = sum_i c_i df_i, u = j / rho          (Eq. 7; sum_i c_i w_i = 0)
//   df_i^eq = w_i [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)]   (Eq. 5)
#pragma once
#include "lattice.cuh"
#include "xlb_types.h"

namespace xlb {

enum Collision { COLL_NONE = 0, COLL_BGK = 1, COLL_KBC = 2 };

// Periodic neighbour coordinates of one cell: xo[k] = x + k - 1 wrapped, and
// rb[b][c] = row offset of (y + b - 1, z + c - 1) wrapped.  The source of
// direction i is xo[1 - cx] + rb[1 - cy][1 - cz].  Cell indices are 32-bit
// (the library caps a lattice at 2^31 - 1 cells); plane offsets are 64-bit.
struct Nbr {
  int xo[3];
  int rb[3][3];
};

__device__ __forceinline__ int wrap_m(int v, int n) { return v == 0 ? n - 1 : v - 1; }
__device__ __forceinline__ int wrap_p(int v, int n) { return v == n - 1 ? 0 : v + 1; }

__device__ __forceinline__ void make_nbr(Nbr& nb, int x, int y, int z, int nx, int ny, int nz) {
  nb.xo[0] = wrap_m(x, nx);
  nb.xo[1] = x;
  nb.xo[2] = wrap_p(x, nx);
  const int ys[3] = {wrap_m(y, ny), y, wrap_p(y, ny)};
  const int zs[3] = {nz > 1 ? wrap_m(z, nz) : 0, z, nz > 1 ? wrap_p(z, nz) : 0};
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) nb.rb[b][c] = nx * (ys[b] + ny * zs[c]);
}

template <int Q>
__device__ __forceinline__ int src_index(const Nbr& nb, int i) {
  return nb.xo[1 - Lattice<Q>::c(i, 0)] + nb.rb[1 - Lattice<Q>::c(i, 1)][1 - Lattice<Q>::c(i, 2)];
}

template <int Q>
__device__ __forceinline__ void moments(const float (&df)[Q], float& drho, float (&j)[3]) {
  drho = 0.f;
  j[0] = j[1] = j[2] = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    drho += df[i];
    if (Lattice<Q>::c(i, 0)) j[0] += Lattice<Q>::c(i, 0) * df[i];
    if (Lattice<Q>::c(i, 1)) j[1] += Lattice<Q>::c(i, 1) * df[i];
    if (Lattice<Q>::c(i, 2)) j[2] += Lattice<Q>::c(i, 2) * df[i];
  }
}

// Moments of order 0, 1 and 2 of the deviations in one pass over the pairs
// (i, opp(i)): their sum carries the even moments, their difference the odd.
// M = sum_i c_ia c_ib df_i, stored xx yy zz xy xz yz.
template <int Q>
__device__ __forceinline__ void moments_kbc(const float (&df)[Q], float& drho, float (&j)[3], float (&M)[6]) {
  drho = df[0];
  j[0] = j[1] = j[2] = 0.f;
#pragma unroll
  for (int a = 0; a < 6; ++a) M[a] = 0.f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (opposite<Q>(i) > i) {
      const float sp = df[i] + df[opposite<Q>(i)], dm = df[i] - df[opposite<Q>(i)];
      constexpr int D = Lattice<Q>::D;
      const int cx = Lattice<Q>::c(i, 0), cy = Lattice<Q>::c(i, 1), cz = D == 3 ? Lattice<Q>::c(i, 2) : 0;
      drho += sp;
      if (cx) j[0] += cx * dm;
      if (cy) j[1] += cy * dm;
      if (cz) j[2] += cz * dm;
      if (cx) M[0] += sp;
      if (cy) M[1] += sp;
      if (cz) M[2] += sp;
      if (cx * cy) M[3] += (float)(cx * cy) * sp;
      if (cx * cz) M[4] += (float)(cx * cz) * sp;
      if (cy * cz) M[5] += (float)(cy * cz) * sp;
    }
  }
}

// Bracket of Eq. 5 without the leading 1: 3 c.u + 4.5 (c.u)^2 - 1.5 u.u
template <int Q>
__device__ __forceinline__ float eq_poly(int i, const float (&u)[3], float usq) {
  float cu = 0.f;
  if (Lattice<Q>::c(i, 0)) cu += Lattice<Q>::c(i, 0) * u[0];
  if (Lattice<Q>::c(i, 1)) cu += Lattice<Q>::c(i, 1) * u[1];
  if (Lattice<Q>::c(i, 2)) cu += Lattice<Q>::c(i, 2) * u[2];
  return cu * (3.0f + 4.5f * cu) - 1.5f * usq;
}

// c_i . u
template <int Q>
__device__ __forceinline__ float cdot(int i, const float (&u)[3]) {
  float cu = 0.f;
  if (Lattice<Q>::c(i, 0)) cu += Lattice<Q>::c(i, 0) * u[0];
  if (Lattice<Q>::c(i, 1)) cu += Lattice<Q>::c(i, 1) * u[1];
  if (Lattice<Q>::c(i, 2)) cu += Lattice<Q>::c(i, 2) * u[2];
  return cu;
}

// Pull: df_i(x) = h_i(x - c_i), periodic (Eq. 2).  Sources on a boundary face
// (StepParams::face) take the rule instead, chosen before any load so that
// each direction is still exactly one load:
//   WALL: h_opp(i)(x);  LID: h_opp(i)(x) + 2 w_i rho_w (c_i . u_w) / cs^2;
//   EQ: f_i^eq(rho_w, u_w) (no load);  FWALL: the plain pull.
// WALL / LID / EQ sources elsewhere hold ghost values (k_boundary).

// Face type of the source coordinate index k (0: v - 1, 1: v, 2: v + 1) on
// one axis: lo / hi are the face types of coordinate 0 and n - 1.
__device__ __forceinline__ int face_code(int v, int n) {
  return (v == 0 ? 1 : 0) | (v == n - 1 ? 2 : 0);
}

// Rule a source takes, from the three axes' face types of its coordinates:
// WALL wins; then a source on an FWALL plane is pulled plainly (0); else LID
// / EQ (at most one of the two meets; verified on the host).  FW = false
// compiles the form for lattices without FWALL faces.
template <bool FW = true>
__device__ __forceinline__ int face_combine(int a, int b, int c) {
  if (a == WALL || b == WALL || c == WALL) return WALL;
  if (FW && (a == FWALL || b == FWALL || c == FWALL)) return 0;
  return a | b | c;
}

// Full-way bounce-back (Section 3.5): the collision of an FWALL cell sends
// every population back where it came from, f*_i = f_opp(i).
template <int Q>
__device__ __forceinline__ void reverse_populations(float (&df)[Q]) {
#pragma unroll
  for (int i = 1; i < Q; ++i)
    if (i < opposite<Q>(i)) {
      const float t = df[i];
      df[i] = df[opposite<Q>(i)];
      df[opposite<Q>(i)] = t;
    }
}

// Returns, with FW, whether the cell itself lies on an FWALL face plane (its
// own coordinates then count as near a face, so that only warps holding such
// cells evaluate it).
// With `outlet` (a cell of an OUTLET plane x = nx - 1 that copies the pull of
// x - 1 in the directions c_x = -1, nb.xo[2] then being x itself) the face
// rules of those directions take the populations of x - 1.
template <int Q, typename S, bool FW = true>
__device__ __forceinline__ bool pull_periodic(const S* __restrict__ src, const StepParams& p, const Nbr& nb,
                                              int self, int x, int y, int z, float (&df)[Q], bool outlet = false) {
  int fcx[3] = {0, 0, 0}, fcy[3] = {0, 0, 0}, fcz[3] = {0, 0, 0};
  bool near = false;
  if (p.has_faces) {
    const int xs[3] = {nb.xo[0], x, nb.xo[2]};
    if (y > 1 && y < p.ny - 2 && (p.nz == 1 || (z > 1 && z < p.nz - 2))) {
      // a row two or more planes from the y / z face planes (uniform over a
      // warp) can only meet x-faces
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int cx = face_code(xs[k], p.nx);
        fcx[k] = (cx & 1 ? p.face[0] : 0) | (cx & 2 ? p.face[1] : 0);
        near |= (k != 1 || FW) && fcx[k];
      }
    } else {
      const int ys[3] = {wrap_m(y, p.ny), y, wrap_p(y, p.ny)};
      const int zs[3] = {p.nz > 1 ? wrap_m(z, p.nz) : 0, z, p.nz > 1 ? wrap_p(z, p.nz) : 0};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int cx = face_code(xs[k], p.nx), cy = face_code(ys[k], p.ny), cz = face_code(zs[k], p.nz);
        fcx[k] = (cx & 1 ? p.face[0] : 0) | (cx & 2 ? p.face[1] : 0);
        fcy[k] = (cy & 1 ? p.face[2] : 0) | (cy & 2 ? p.face[3] : 0);
        fcz[k] = p.nz > 1 ? ((cz & 1 ? p.face[4] : 0) | (cz & 2 ? p.face[5] : 0)) : 0;
        near |= (k != 1 || FW) && (fcx[k] | fcy[k] | fcz[k]);
      }
    }
  }
  const S* base = src;
  // warp-uniform choice: a warp with no lane next to a face loads plainly;
  // otherwise every lane picks each address branch-free, so either way the
  // warp issues one round of Q independent loads
  if (!__any_sync(__activemask(), near)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      df[i] = Store<S>::ld(base + src_index<Q>(nb, i));
      base += p.plane;
    }
    return false;
  }
  // all loads first (addresses chosen branch-free), adjustments after, so
  // the Q loads stay in flight together
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int t = i == 0 ? 0
                         : face_combine<FW>(fcx[1 - Lattice<Q>::c(i, 0)], fcy[1 - Lattice<Q>::c(i, 1)],
                                            fcz[1 - Lattice<Q>::c(i, 2)]);
    const int own = (Lattice<Q>::c(i, 0) == -1 && outlet) ? self - 1 : self;
    const S* a = t ? src + (long long)opposite<Q>(i) * p.plane + own : base + src_index<Q>(nb, i);
    df[i] = Store<S>::ld(a);
    base += p.plane;
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int t = face_combine<FW>(fcx[1 - Lattice<Q>::c(i, 0)], fcy[1 - Lattice<Q>::c(i, 1)],
                                   fcz[1 - Lattice<Q>::c(i, 2)]);
    if (t == EQ) df[i] = p.eq_df[i];
    if (t == LID) df[i] += p.lid_term[i];
  }
  // where a WALL face meets an FWALL plane the cell is WALL and its slots are
  // never read, so reversing it as well is harmless
  return FW && (fcx[1] == FWALL || fcy[1] == FWALL || fcz[1] == FWALL);
}

// Velocity boundaries at INLET cells, with inward normal n = sign e_axis
// (StepParams::inlet_axis / inlet_sign; +x, an inflow, by default; with a
// velocity parallel to the wall they are a moving wall).  The unknown
// populations are those entering the fluid through the boundary, c_i.n = +1.
// The velocity is StepParams::inlet_u, or the cell's entry of
// StepParams::inlet_field (a velocity profile) when that is set.
template <int Q>
__device__ __forceinline__ void inlet_velocity(const StepParams& p, int self, float (&u)[3]) {
  u[0] = p.inlet_u[0];
  u[1] = p.inlet_u[1];
  u[2] = p.inlet_u[2];
  if (p.inlet_field) {
    const long long n = (long long)p.nx * p.ny * p.nz;
    u[0] = p.inlet_field[self];
    u[1] = p.inlet_field[n + self];
    u[2] = Lattice<Q>::D == 3 ? p.inlet_field[2 * n + self] : 0.f;
  }
}

// c_i . n for the inlet normal
template <int Q>
__device__ __forceinline__ int inlet_cn(const StepParams& p, int i) {
  const int c = p.inlet_axis == 0 ? Lattice<Q>::c(i, 0) : (p.inlet_axis == 1 ? Lattice<Q>::c(i, 1) : Lattice<Q>::c(i, 2));
  return p.inlet_sign * c;
}

// rho = [sum_{c.n=0} f_i + 2 sum_{c.n=-1} f_i] / (1 - u.n); in deviations the
// rest parts of the numerator sum to exactly 1.
template <int Q>
__device__ __forceinline__ float inlet_density(const StepParams& p, const float (&df)[Q], const float (&u)[3]) {
  float s = 1.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cn = inlet_cn<Q>(p, i);
    if (cn == 0) s += df[i];
    if (cn == -1) s += 2.0f * df[i];
  }
  const float un = p.inlet_sign * (p.inlet_axis == 0 ? u[0] : (p.inlet_axis == 1 ? u[1] : u[2]));
  return s / (1.0f - un);
}

// Zou-He: each unknown f_i = f_opp(i) + f_i^eq - f_opp(i)^eq = f_opp(i) + 6 w_i rho (c_i . u).
template <int Q>
__device__ __forceinline__ void zou_he_inlet(const StepParams& p, int self, float (&df)[Q]) {
  float u[3];
  inlet_velocity<Q>(p, self, u);
  const float rho = inlet_density<Q>(p, df, u);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (inlet_cn<Q>(p, i) == 1) {
      float cu = Lattice<Q>::c(i, 0) * u[0] + Lattice<Q>::c(i, 1) * u[1];
      if (Lattice<Q>::D == 3) cu += Lattice<Q>::c(i, 2) * u[2];
      df[i] = df[opposite<Q>(i)] + 6.0f * weight<Q>(i) * rho * cu;
    }
  }
}

// Regularized velocity boundary (Latt et al. 2008; the other inflow rule
// Section 4.3 names, and the regularized lid of Section 4.2): rho as for
// Zou-He; non-equilibrium parts of the known populations, those of the
// unknown ones by bounce-back; Pi = sum_i c_i c_i f^neq_i; every population
// becomes f_i = f_i^eq(rho, u) + w_i / (2 cs^4) (c_i c_i - cs^2 I) : Pi.
template <int Q>
__device__ __forceinline__ void regularized_inlet(const StepParams& p, int self, float (&df)[Q]) {
  float u[3];
  inlet_velocity<Q>(p, self, u);
  const float rho = inlet_density<Q>(p, df, u);
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  // equilibrium deviations f_i^eq - w_i, then the non-equilibrium parts
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float eqd = weight<Q>(i) * (rho - 1.0f) + weight<Q>(i) * rho * eq_poly<Q>(i, u, usq);
    df[i] -= eqd;  // df now holds f^neq_i
  }
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (inlet_cn<Q>(p, i) == 1) df[i] = df[opposite<Q>(i)];
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cx = Lattice<Q>::c(i, 0), cy = Lattice<Q>::c(i, 1), cz = Lattice<Q>::c(i, 2);
    pxx += cx * cx * df[i];
    pyy += cy * cy * df[i];
    pzz += cz * cz * df[i];
    pxy += cx * cy * df[i];
    pxz += cx * cz * df[i];
    pyz += cy * cz * df[i];
  }
  constexpr float cs2 = 1.0f / 3.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cx = Lattice<Q>::c(i, 0), cy = Lattice<Q>::c(i, 1), cz = Lattice<Q>::c(i, 2);
    float qpi = (cx * cx - cs2) * pxx + (cy * cy - cs2) * pyy + 2.0f * cx * cy * pxy;
    if (Lattice<Q>::D == 3) qpi += (cz * cz - cs2) * pzz + 2.0f * (cx * cz * pxz + cy * cz * pyz);
    const float eqd = weight<Q>(i) * (rho - 1.0f) + weight<Q>(i) * rho * eq_poly<Q>(i, u, usq);
    df[i] = eqd + 4.5f * weight<Q>(i) * qpi;  // 1 / (2 cs^4) = 4.5
  }
}

// The velocity boundary of an INLET cell, by the chosen scheme.
template <int Q>
__device__ __forceinline__ void inlet_rule(const StepParams& p, int self, float (&df)[Q]) {
  if (p.inlet_regularized)
    regularized_inlet<Q>(p, self, df);
  else
    zou_he_inlet<Q>(p, self, df);
}

// Post-stream populations of a fluid-like or FWALL cell.  The pull applies
// the face rules and reads the ghost values that every other WALL / LID / EQ
// source carries (see k_boundary), i.e. the bounce-back, moving-wall and
// equilibrium rules; INLET cells then rebuild their c_x = +1 populations by
// Zou-He and OUTLET cells copy their c_x = -1 populations from the pull at
// x - 1 (zero-gradient outflow).
template <int Q, typename S>
__device__ __forceinline__ void pull_cell(const S* __restrict__ src, const StepParams& p, int x, int y, int z,
                                          int type, const Nbr& nb, float (&df)[Q]) {
  const int self = x + p.nx * (y + p.ny * z);
  pull_periodic<Q, S>(src, p, nb, self, x, y, z, df);
  if (type == INLET) inlet_rule<Q>(p, self, df);
  if (type == OUTLET) {
    const int xl = wrap_m(x, p.nx);
    Nbr nl;
    make_nbr(nl, xl, y, z, p.nx, p.ny, p.nz);
    float dl[Q];
    pull_periodic<Q, S>(src, p, nl, self - x + xl, xl, y, z, dl);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (Lattice<Q>::c(i, 0) == -1) df[i] = dl[i];
  }
}

// The collision code below walks the rest direction and the pairs
// (i, opp(i)), i < opp(i): with a = 3 c_i.u and b = 4.5 (c_i.u)^2 - 1.5 u.u
// the bracket of Eq. 5 is b + a for i and b - a for opp(i), and every even
// function of c (the KBC shear part, the second moments) is shared.

// Exact-difference body force: df_i += f_i^eq(rho, u + F/rho) - f_i^eq(rho, u).
template <int Q>
__device__ __forceinline__ void add_force(float (&df)[Q], float rho, const float (&u)[3], float usq,
                                          const float (&F)[3]) {
  const float ir = 1.0f / rho;
  float v[3] = {u[0] + F[0] * ir, u[1] + F[1] * ir, u[2] + F[2] * ir};
  if (Lattice<Q>::D == 2) v[2] = 0.f;
  const float vsq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const float dsq = -1.5f * (vsq - usq);
  df[0] += weight<Q>(0) * rho * dsq;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (opposite<Q>(i) > i) {
      const float cu = cdot<Q>(i, u), cv = cdot<Q>(i, v);
      const float e = 4.5f * (cv * cv - cu * cu) + dsq, o = 3.0f * (cv - cu);
      const float wr = weight<Q>(i) * rho;
      df[i] += wr * (e + o);
      df[opposite<Q>(i)] += wr * (e - o);
    }
  }
}

// KBC shear population ds_i from hd = D_aa / 2 (a = x, y, z) and
// qo = Pi_ab / 4 (ab = xy, xz, yz); zero on the rest and corner directions.
template <int Q>
__device__ __forceinline__ float kbc_ds(int i, const float (&hd)[3], const float (&qo)[3]) {
  const int cx = Lattice<Q>::c(i, 0), cy = Lattice<Q>::c(i, 1), cz = Lattice<Q>::c(i, 2);
  if (nnz<Q>(i) == 1) return cx ? hd[0] : (cy ? hd[1] : hd[2]);
  if (nnz<Q>(i) == 2) {
    if (cx && cy) return (float)(cx * cy) * qo[0];
    if (cx && cz) return (float)(cx * cz) * qo[1];
    return (float)(cy * cz) * qo[2];
  }
  return 0.f;
}

// Collision C of Eq. 1 on one fluid-like cell, in place on deviations.
//   BGK (Eq. 3): df_i += omega (df_i^eq - df_i)
//   KBC (Karlin, Bosch, Chikatamarla 2014): f^neq = ds + dh, beta = omega / 2,
//     gamma = 1/beta - (2 - 1/beta) <ds|dh> / <dh|dh>,  <a|b> = sum a_i b_i / f_i^eq,
//     f_i <- f_i - beta (2 ds_i + gamma dh_i)
//   where ds carries the deviatoric second moments of f^neq on the natural
//   moment basis: ds_i = D_aa / 2 for c_i = +-e_a, ds_i = c_ia c_ib Pi_ab / 4
//   for c_i with two non-zero components a, b, and 0 otherwise
//   (D_aa = Pi_aa - tr(Pi) / d).
template <int Q, int COLL>
__device__ __forceinline__ void collide(float (&df)[Q], const StepParams& p) {
  if (COLL == COLL_NONE) return;
  float drho, j[3], M[6];
  if (COLL == COLL_KBC)
    moments_kbc<Q>(df, drho, j, M);
  else
    moments<Q>(df, drho, j);
  const float rho = 1.0f + drho;
  const float ir = 1.0f / rho;
  float u[3] = {j[0] * ir, j[1] * ir, j[2] * ir};
  if (Lattice<Q>::D == 2) u[2] = 0.f;
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  float force_u[3];
  if (p.has_force) {
    force_u[0] = u[0];
    force_u[1] = u[1];
    force_u[2] = u[2];
  }
  const float b0 = -1.5f * usq;  // b of the rest direction (c = 0)
  if (COLL == COLL_BGK) {
    df[0] = fmaf(p.omega, weight<Q>(0) * (drho + rho * b0) - df[0], df[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (opposite<Q>(i) > i) {
        const int j = opposite<Q>(i);
        const float cu = cdot<Q>(i, u);
        const float bb = drho + rho * fmaf(4.5f * cu, cu, b0), ra = rho * 3.0f * cu;
        const float w = weight<Q>(i);
        df[i] = fmaf(p.omega, w * (bb + ra) - df[i], df[i]);
        df[j] = fmaf(p.omega, w * (bb - ra) - df[j], df[j]);
      }
    }
  } else {
    // KBC.  The second moments of f^neq come from those of the deviations
    // (moments_kbc) and the closed form of the equilibrium's: on these
    // lattices sum_i c_ia c_ib f_i^eq = rho (d_ab / 3 + u_a u_b), so
    //   P_ab = M_ab - rho u_a u_b - d_ab drho / 3.
    // One pass then turns df into f^neq and forms <ds|dh> and <dh|dh>, with
    // dh = f^neq - ds; with them the update reads
    //   df_i <- df_i^eq + (1 - beta gamma) f^neq_i - beta (2 - gamma) ds_i.
    constexpr float third = 1.0f / 3.0f;
    const float dd = drho * third;
    const float P0 = M[0] - rho * u[0] * u[0] - dd, P1 = M[1] - rho * u[1] * u[1] - dd;
    const float P2 = Lattice<Q>::D == 3 ? M[2] - rho * u[2] * u[2] - dd : 0.f;
    constexpr float inv_d = 1.0f / Lattice<Q>::D;
    const float tr = (P0 + P1 + P2) * inv_d;
    // ds_i: D_aa / 2 on the axis directions, c_a c_b Pi_ab / 4 on the two-component ones
    const float hd[3] = {0.5f * (P0 - tr), 0.5f * (P1 - tr), 0.5f * (P2 - tr)};
    const float qo[3] = {0.25f * (M[3] - rho * u[0] * u[1]), 0.25f * (M[4] - rho * u[0] * u[2]),
                         0.25f * (M[5] - rho * u[1] * u[2])};
    // <a|b> = sum a_i b_i / f_i^eq with f_i^eq = w_i rho (1 + b +- a); the
    // common 1/rho cancels in gamma, and one reciprocal serves a pair:
    // 1 / (X +- a) = (X -+ a) / (X^2 - a^2).  The rest direction has ds = 0.
    df[0] -= weight<Q>(0) * (drho + rho * b0);
    float hh = df[0] * df[0] * __fdividef(1.0f / weight<Q>(0), 1.0f + b0), sh = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (opposite<Q>(i) > i) {
        const int j = opposite<Q>(i);
        const float cu = cdot<Q>(i, u);
        const float w = weight<Q>(i);
        const float bq = fmaf(4.5f * cu, cu, b0), a3 = 3.0f * cu;
        const float bb = drho + rho * bq, ra = rho * a3;
        const float fi = df[i] - w * (bb + ra), fj = df[j] - w * (bb - ra);
        df[i] = fi;
        df[j] = fj;
        const float X = 1.0f + bq;
        const float rc = __fdividef(1.0f / w, fmaf(X, X, -a3 * a3));
        const float ri = (X - a3) * rc, rj = (X + a3) * rc;
        const float s_ = kbc_ds<Q>(i, hd, qo);
        const float hi = fi - s_, hj = fj - s_;
        if (nnz<Q>(i) < 3) sh = fmaf(s_, fmaf(hi, ri, hj * rj), sh);
        hh = fmaf(hi * hi, ri, fmaf(hj * hj, rj, hh));
      }
    }
    const float beta = 0.5f * p.omega;
    const float ib = 1.0f / beta;
    const float gamma = (hh < 1e-20f * rho) ? 2.0f : ib - (2.0f - ib) * sh / hh;
    const float a1 = 1.0f - beta * gamma, a2 = beta * (2.0f - gamma);
    df[0] = fmaf(a1, df[0], weight<Q>(0) * (drho + rho * b0));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (opposite<Q>(i) > i) {
        const int j = opposite<Q>(i);
        const float cu = cdot<Q>(i, u);
        const float w = weight<Q>(i);
        const float bb = drho + rho * fmaf(4.5f * cu, cu, b0), ra = rho * 3.0f * cu;
        const float sd = a2 * kbc_ds<Q>(i, hd, qo);
        df[i] = fmaf(w, bb + ra, fmaf(a1, df[i], -sd));
        df[j] = fmaf(w, bb - ra, fmaf(a1, df[j], -sd));
      }
    }
  }
  if (p.has_force) add_force<Q>(df, rho, force_u, usq, p.F);
}

}  // namespace xlb
