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
  __device__ __forceinline__ static void st_stream(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
};

template <>
struct Store<__nv_bfloat16> {
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ __forceinline__ static float ld_l2(const __nv_bfloat16* p) { return __bfloat162float(__ldcg(p)); }
  __device__ __forceinline__ static void st_l2(__nv_bfloat16* p, float v) { __stcg(p, __float2bfloat16_rn(v)); }
  __device__ __forceinline__ static float ld_plain(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ __forceinline__ static void st_stream(__nv_bfloat16* p, float v) {
    __stcs(p, __float2bfloat16_rn(v));
  }
};

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

// 16-bit storage: V = 8 (one 16-byte word group) or V = 4 (8 bytes)
template <typename H, int V>
struct VecIO16 {
  static constexpr int W = V / 2;  // 32-bit words
  using O = Half2Ops<H>;
  __device__ __forceinline__ static void ld(const H* p, float (&v)[V]) {
    uint32_t w[W];
    if (W == 4) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
      w[0] = q.x; w[1] = q.y; if (W == 4) { w[2 % W] = q.z; w[3 % W] = q.w; }
    } else {
      const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
      w[0] = q.x; w[1 % W] = q.y;
    }
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
    if (W == 4)
      *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1 % W], w[2 % W], w[3 % W]);
    else
      *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1 % W]);
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

}  // namespace xlb
