// Lattice-independent kernels: mask preparation and the final FP64
// reduction of block partial sums.
#include <cuda_runtime.h>

#include "launch.h"
#include "lattice.cuh"

namespace xlb {

long long row_blocks(const StepParams& p) {
  const long long nxb = (p.nx + 127) / 128;
  return nxb * (long long)p.ny * p.nz;
}

// flags = type | FLAG_SLOW where a fluid-like cell has a non-fluid-like cell
// in its Q-stencil, or is an INLET / OUTLET cell.  Codes >= 6 set *err.
template <int Q>
__global__ void k_mask_prepare(const uint8_t* __restrict__ mask, uint8_t* __restrict__ flags, int nx, int ny,
                               int nz, int* err) {
  const long long n = (long long)nx * ny * nz;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    const int t = mask[cell];
    if (t > EQ) {
      atomicExch(err, 1);
      flags[cell] = WALL;
      continue;
    }
    int slow = (t == INLET || t == OUTLET);
    if (fluid_like(t) && !slow) {
      const int x = (int)(cell % nx);
      const long long r = cell / nx;
      const int y = (int)(r % ny);
      const int z = (int)(r / ny);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        int xs = x - Lattice<Q>::c(i, 0), ys = y - Lattice<Q>::c(i, 1), zs = z - Lattice<Q>::c(i, 2);
        xs = xs < 0 ? nx - 1 : (xs >= nx ? 0 : xs);
        ys = ys < 0 ? ny - 1 : (ys >= ny ? 0 : ys);
        zs = zs < 0 ? nz - 1 : (zs >= nz ? 0 : zs);
        const int ts = mask[xs + (long long)nx * (ys + (long long)ny * zs)];
        if (!fluid_like(ts)) slow = 1;
      }
    }
    flags[cell] = (uint8_t)(t | (slow ? FLAG_SLOW : 0));
  }
}

int launch_mask_prepare(int Q, const uint8_t* mask, uint8_t* flags, int nx, int ny, int nz, int* err,
                        void* stream) {
  const long long n = (long long)nx * ny * nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  if (blocks < 1) blocks = 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (Q == 9)
    k_mask_prepare<9><<<(unsigned)blocks, 256, 0, s>>>(mask, flags, nx, ny, nz, err);
  else if (Q == 19)
    k_mask_prepare<19><<<(unsigned)blocks, 256, 0, s>>>(mask, flags, nx, ny, nz, err);
  else if (Q == 27)
    k_mask_prepare<27><<<(unsigned)blocks, 256, 0, s>>>(mask, flags, nx, ny, nz, err);
  else
    return -1;
  return 0;
}

// Sums n rows of 4 doubles in a fixed order (deterministic): each thread
// strides over rows, then a fixed shared-memory tree.
__global__ void k_reduce_final(const double* __restrict__ partial, long long n, double* out) {
  __shared__ double s[4][256];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long r = threadIdx.x; r < n; r += blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] += partial[4 * r + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 4; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

int launch_reduce_final(const double* partial, long long n, double* out, void* stream) {
  k_reduce_final<<<1, 256, 0, (cudaStream_t)stream>>>(partial, n, out);
  return 0;
}

}  // namespace xlb
