// Lattice velocity sets, weights and population storage types of the GPU path.
//
// Velocity order: rest first, then the order of the paper's Figure 1 (the
// D2Q9 / D3Q19 / D3Q27 diagrams, Section 2).  Weights by |c|^2 are the
// standard ones (the paper does not print them): D2Q9 4/9, 1/9, 1/36;
// D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.
//
// Every loop over directions in the kernels is fully unrolled, so these
// constexpr lookups fold to immediates.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace xlb {

template <int Q>
struct Lattice;

template <>
struct Lattice<9> {
  static constexpr int D = 2;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {1, -1, 0}, {-1, 1, 0},  {-1, -1, 0}};
    return t[i][a];
  }
};

template <>
struct Lattice<19> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},   {1, 0, 0},  {0, 1, 0},   {0, 0, 1},   {-1, 0, 0},
                              {0, -1, 0},  {0, 0, -1}, {1, 1, 0},   {1, -1, 0},  {-1, 1, 0},
                              {-1, -1, 0}, {1, 0, 1},  {1, 0, -1},  {-1, 0, 1},  {-1, 0, -1},
                              {0, 1, 1},   {0, 1, -1}, {0, -1, 1},  {0, -1, -1}};
    return t[i][a];
  }
};

template <>
struct Lattice<27> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[27][3] = {{0, 0, 0},   {1, 0, 0},   {0, 1, 0},   {0, 0, 1},   {-1, 0, 0},
                              {0, -1, 0},  {0, 0, -1},  {1, 1, 0},   {1, -1, 0},  {-1, 1, 0},
                              {-1, -1, 0}, {1, 0, 1},   {1, 0, -1},  {-1, 0, 1},  {-1, 0, -1},
                              {0, 1, 1},   {0, 1, -1},  {0, -1, 1},  {0, -1, -1}, {1, 1, 1},
                              {1, 1, -1},  {1, -1, 1},  {1, -1, -1}, {-1, 1, 1},  {-1, 1, -1},
                              {-1, -1, 1}, {-1, -1, -1}};
    return t[i][a];
  }
};

// |c_i|^2
template <int Q>
__host__ __device__ constexpr int csq(int i) {
  return Lattice<Q>::c(i, 0) * Lattice<Q>::c(i, 0) + Lattice<Q>::c(i, 1) * Lattice<Q>::c(i, 1) +
         Lattice<Q>::c(i, 2) * Lattice<Q>::c(i, 2);
}

// number of non-zero velocity components of c_i
template <int Q>
__host__ __device__ constexpr int nnz(int i) {
  return (Lattice<Q>::c(i, 0) != 0) + (Lattice<Q>::c(i, 1) != 0) + (Lattice<Q>::c(i, 2) != 0);
}

template <int Q>
__host__ __device__ constexpr double weight_d(int i) {
  return Q == 9 ? (csq<Q>(i) == 0 ? 4.0 / 9.0 : csq<Q>(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0)
       : Q == 19 ? (csq<Q>(i) == 0 ? 1.0 / 3.0 : csq<Q>(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0)
                 : (csq<Q>(i) == 0 ? 8.0 / 27.0
                    : csq<Q>(i) == 1 ? 2.0 / 27.0
                    : csq<Q>(i) == 2 ? 1.0 / 54.0
                                     : 1.0 / 216.0);
}

template <int Q>
__host__ __device__ constexpr float weight(int i) {
  return (float)weight_d<Q>(i);
}

template <int Q>
__host__ __device__ constexpr int opposite(int i) {
  int r = 0;
  for (int k = 0; k < Q; ++k)
    if (Lattice<Q>::c(k, 0) == -Lattice<Q>::c(i, 0) && Lattice<Q>::c(k, 1) == -Lattice<Q>::c(i, 1) &&
        Lattice<Q>::c(k, 2) == -Lattice<Q>::c(i, 2))
      r = k;
  return r;
}

// ---------------------------------------------------------------------------
// Population storage.  Every storage type holds the deviation
// df_i = f_i - w_i rho0 (rho0 = 1) of a population from the rest state; the
// arithmetic is FP32 throughout.  FP16 / BF16 stores round to nearest even.

template <typename S>
struct Store;

// ld_l2 / st_l2: coherent at L2 (bypass L1), for data written earlier in the
// same kernel by other threads of the block.
template <>
struct Store<float> {
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static float ld_l2(const float* p) { return __ldcg(p); }
  __device__ __forceinline__ static void st_l2(float* p, float v) { __stcg(p, v); }
  __device__ __forceinline__ static float ld_plain(const float* p) { return *p; }
  __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
  __device__ __forceinline__ static void st_stream(float* p, float v) { __stcs(p, v); }
};

template <>
struct Store<__half> {
  __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ __forceinline__ static float ld_l2(const __half* p) { return __half2float(__ldcg(p)); }
  __device__ __forceinline__ static void st_l2(__half* p, float v) { __stcg(p, __float2half_rn(v)); }
  __device__ __forceinline__ static float ld_plain(const __half* p) { return __half2float(*p); }
  __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
  __device__ __forceinline__ static __half cvt(float v) { return __float2half_rn(v); }
  __device__ __forceinline__ static void st_stream(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
};

template <>
struct Store<__nv_bfloat16> {
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ __forceinline__ static float ld_l2(const __nv_bfloat16* p) { return __bfloat162float(__ldcg(p)); }
  __device__ __forceinline__ static void st_l2(__nv_bfloat16* p, float v) { __stcg(p, __float2bfloat16_rn(v)); }
  __device__ __forceinline__ static float ld_plain(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ __forceinline__ static __nv_bfloat16 cvt(float v) { return __float2bfloat16_rn(v); }
  __device__ __forceinline__ static void st_stream(__nv_bfloat16* p, float v) {
    __stcs(p, __float2bfloat16_rn(v));
  }
};

// ---------------------------------------------------------------------------
// Rounding of one cell's post-collision populations into the storage type.
//
// FP32 stores the value; FP16 rounds to nearest even.  BF16 (8 significant
// bits) rounds stochastically: round-to-nearest-even makes the rounding error
// a fixed function of the value, so on a smooth flow neighbouring cells err
// alike and the error builds up coherently (Taylor-Green 128^2, 1000 steps:
// relative velocity error 7e-3 to 8e-3 against the FP64 result); rounding up
// with probability equal to the discarded fraction makes the error zero-mean
// and spatially uncorrelated, and viscosity damps it (3e-3 on the same run).
// The random bits come from a hash of the cell index and the FP32 bits of
// all the cell's values, so a run is reproducible, every kernel variant
// rounds a given cell identically, and graph replays need no step counter:
//   s_0 = fmix32(cell * 0x9E3779B9 ^ (xor of the Q values' bits)),
// fmix32 being the 32-bit finaliser of MurmurHash3 (Appleby, public domain);
// direction i takes the high 16 bits of s_{i+1}, where s_{k+1} = a s_k + c
// is the 32-bit LCG of PCG (O'Neill 2014; a = 747796405, c = 2891336453),
// jumped to step i + 1 directly (s_{i+1} = A_i s_0 + C_i); the value's FP32
// bit pattern plus those 16 bits, truncated to its high half, is the BF16.
// Non-finite values round to nearest even.

__host__ __device__ constexpr uint32_t lcg_jump_mul(int i) {
  uint32_t m = 747796405u;
  for (int k = 0; k < i; ++k) m *= 747796405u;
  return m;
}
__host__ __device__ constexpr uint32_t lcg_jump_add(int i) {
  uint32_t c = 2891336453u;
  for (int k = 0; k < i; ++k) c = c * 747796405u + 2891336453u;
  return c;
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// BF16 bits of v rounded up with probability (discarded bits) / 2^16, given
// 16 random bits r.
__device__ __forceinline__ uint16_t bf16_stochastic_bits(float v, uint32_t r) {
  const uint32_t b = __float_as_uint(v);
  if ((b & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  return (uint16_t)((b + r) >> 16);
}

template <typename S>
struct CellRound {
  template <int Q>
  __device__ __forceinline__ void begin(uint32_t, const float (&)[Q]) {}
  __device__ __forceinline__ void st(S* p, int, float v) const { Store<S>::st(p, v); }
  __device__ __forceinline__ void st_l2(S* p, int, float v) const { Store<S>::st_l2(p, v); }
  // the stored value as the 16-bit pattern (16-bit storage only)
  __device__ __forceinline__ uint16_t bits(int, float v) const {
    const S h = Store<S>::cvt(v);
    uint16_t u;
    memcpy(&u, &h, 2);
    return u;
  }
  // the value as it reads back after the store
  __device__ __forceinline__ float rounded(int, float v) const {
    S h;
    Store<S>::st(&h, v);
    return Store<S>::ld_plain(&h);
  }
};

template <>
struct CellRound<__nv_bfloat16> {
  uint32_t s0;
  template <int Q>
  __device__ __forceinline__ void begin(uint32_t cell, const float (&v)[Q]) {
    uint32_t f = 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i) f ^= __float_as_uint(v[i]);
    s0 = fmix32((cell * 0x9E3779B9u) ^ f);
  }
  __device__ __forceinline__ uint16_t bits(int i, float v) const {
    return bf16_stochastic_bits(v, (lcg_jump_mul(i) * s0 + lcg_jump_add(i)) >> 16);
  }
  __device__ __forceinline__ void st(__nv_bfloat16* p, int i, float v) const {
    *p = __ushort_as_bfloat16(bits(i, v));
  }
  __device__ __forceinline__ float rounded(int i, float v) const {
    return __uint_as_float((uint32_t)bits(i, v) << 16);
  }
  __device__ __forceinline__ void st_l2(__nv_bfloat16* p, int i, float v) const {
    __stcg(p, __ushort_as_bfloat16(bits(i, v)));
  }
};

// A ghost value (the value a boundary rule gives a pull from a solid cell,
// written into that cell's slot): FP32 / FP16 as Store<S>::st; BF16 rounds
// stochastically with random bits hashed from the slot index and the value,
// so that a constant boundary value (an equilibrium lid) is rounded up on a
// fraction of the slots and down on the others instead of the same way
// everywhere.
template <typename S>
__device__ __forceinline__ void st_ghost(S* p, uint32_t, float v) {
  Store<S>::st(p, v);
}
template <>
__device__ __forceinline__ void st_ghost<__nv_bfloat16>(__nv_bfloat16* p, uint32_t key, float v) {
  *p = __ushort_as_bfloat16(bf16_stochastic_bits(v, fmix32(key ^ __float_as_uint(v)) >> 16));
}

// ---------------------------------------------------------------------------
// Vector access to V consecutive stored populations (V * sizeof(S) = 8 or 16
// bytes, naturally aligned), converted to / from FP32.

template <typename S, int V>
struct VecIO;

template <>
struct VecIO<float, 4> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[4]) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
  }
  __device__ __forceinline__ static void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <>
struct VecIO<float, 2> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[2]) {
    const float2 w = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = w.x; v[1] = w.y;
  }
  __device__ __forceinline__ static void st(float* p, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};

template <typename H>
struct Half2Ops;
template <>
struct Half2Ops<__half> {
  using T2 = __half2;
  __device__ __forceinline__ static float2 to_f2(T2 h) { return __half22float2(h); }
  __device__ __forceinline__ static T2 from_f2(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct Half2Ops<__nv_bfloat16> {
  using T2 = __nv_bfloat162;
  __device__ __forceinline__ static float2 to_f2(T2 h) { return __bfloat1622float2(h); }
  __device__ __forceinline__ static T2 from_f2(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

// 16-bit storage: V = 8 (16 bytes), 4 (8 bytes) or 2 (4 bytes), naturally
// aligned.
template <typename H, int V>
struct VecIO16 {
  static constexpr int W = V / 2;  // 32-bit words
  using O = Half2Ops<H>;
  __device__ __forceinline__ static void ld_words(const H* p, uint32_t (&w)[W]) {
    if constexpr (W == 4) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
      w[0] = q.x;
      w[1] = q.y;
      w[2] = q.z;
      w[3] = q.w;
    } else if constexpr (W == 2) {
      const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
      w[0] = q.x;
      w[1] = q.y;
    } else {
      w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
    }
  }
  __device__ __forceinline__ static void st_words(H* p, const uint32_t (&w)[W]) {
    if constexpr (W == 4)
      *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    else if constexpr (W == 2)
      *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    else
      *reinterpret_cast<unsigned int*>(p) = w[0];
  }
  __device__ __forceinline__ static void ld(const H* p, float (&v)[V]) {
    uint32_t w[W];
    ld_words(p, w);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      typename O::T2 h;
      memcpy(&h, &w[k], 4);
      const float2 f = O::to_f2(h);
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
  __device__ __forceinline__ static void st(H* p, const float (&v)[V]) {
    uint32_t w[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const typename O::T2 h = O::from_f2(v[2 * k], v[2 * k + 1]);
      memcpy(&w[k], &h, 4);
    }
    st_words(p, w);
  }
  // store V values already rounded to their 16-bit patterns
  __device__ __forceinline__ static void st_bits(H* p, const uint16_t (&b)[V]) {
    uint32_t w[W];
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = (uint32_t)b[2 * k] | ((uint32_t)b[2 * k + 1] << 16);
    st_words(p, w);
  }
};

template <>
struct VecIO<__half, 8> : VecIO16<__half, 8> {};
template <>
struct VecIO<__half, 4> : VecIO16<__half, 4> {};
template <>
struct VecIO<__nv_bfloat16, 8> : VecIO16<__nv_bfloat16, 8> {};
template <>
struct VecIO<__nv_bfloat16, 4> : VecIO16<__nv_bfloat16, 4> {};
template <>
struct VecIO<__half, 2> : VecIO16<__half, 2> {};
template <>
struct VecIO<__nv_bfloat16, 2> : VecIO16<__nv_bfloat16, 2> {};

}  // namespace xlb
