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

template <>
struct Store<float> {
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static float ld_plain(const float* p) { return *p; }
  __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
  __device__ __forceinline__ static void st_stream(float* p, float v) { __stcs(p, v); }
};

template <>
struct Store<__half> {
  __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ __forceinline__ static float ld_plain(const __half* p) { return __half2float(*p); }
  __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
  __device__ __forceinline__ static void st_stream(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
};

template <>
struct Store<__nv_bfloat16> {
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  __device__ __forceinline__ static float ld_plain(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ __forceinline__ static void st_stream(__nv_bfloat16* p, float v) {
    __stcs(p, __float2bfloat16_rn(v));
  }
};

}  // namespace xlb
