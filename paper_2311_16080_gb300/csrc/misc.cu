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

// Boundary tables, built once per mask in two passes (per-block counts, an
// exclusive scan of the counts on the host, then ordered per-block writes):
//  - links: one entry per (fluid cell x, direction i) whose source cell
//    x - c_i is WALL, LID or EQ, packed as {x, i | type << 8};
//  - fix-up cells: every INLET and OUTLET cell.
constexpr int LIST_BLOCK = 256;

template <int Q>
__device__ __forceinline__ int cell_links(const uint8_t* __restrict__ mask, long long cell, int nx, int ny, int nz,
                                          int* types /* Q or null */) {
  const int x = (int)(cell % nx);
  const long long r = cell / nx;
  const int y = (int)(r % ny), z = (int)(r / ny);
  int n = 0;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int xs = x - Lattice<Q>::c(i, 0), ys = y - Lattice<Q>::c(i, 1), zs = z - Lattice<Q>::c(i, 2);
    xs = xs < 0 ? nx - 1 : (xs >= nx ? 0 : xs);
    ys = ys < 0 ? ny - 1 : (ys >= ny ? 0 : ys);
    zs = zs < 0 ? nz - 1 : (zs >= nz ? 0 : zs);
    const int t = mask[xs + (long long)nx * (ys + (long long)ny * zs)] & FLAG_TYPE;
    const bool link = !fluid_like(t);
    if (types) types[i] = link ? t : 0;
    n += link;
  }
  return n;
}

// Block-wide exclusive scan of one int per thread (LIST_BLOCK threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[LIST_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < LIST_BLOCK / 32; ++w) {
      const int c = warp_sums[w];
      warp_sums[w] = run;
      run += c;
    }
    *total = run;
  }
  __syncthreads();
  return warp_sums[warp] + incl - v;
}

template <int Q>
__global__ void k_bnd_count(const uint8_t* __restrict__ flags, long long n, int nx, int ny, int nz, int* counts) {
  const long long cell = blockIdx.x * (long long)LIST_BLOCK + threadIdx.x;
  int nl = 0, nf = 0;
  if (cell < n) {
    const int t = flags[cell] & FLAG_TYPE;
    if (t == FLUID && (flags[cell] & FLAG_SLOW)) nl = cell_links<Q>(flags, cell, nx, ny, nz, nullptr);
    nf = (t == INLET || t == OUTLET);
  }
  __shared__ int tl, tf;
  block_exclusive_scan(nl, &tl);
  block_exclusive_scan(nf, &tf);
  if (threadIdx.x == 0) {
    counts[2 * blockIdx.x] = tl;
    counts[2 * blockIdx.x + 1] = tf;
  }
}

template <int Q>
__global__ void k_bnd_write(const uint8_t* __restrict__ flags, long long n, int nx, int ny, int nz,
                            const long long* __restrict__ offs, int2* links, int* fix) {
  const long long cell = blockIdx.x * (long long)LIST_BLOCK + threadIdx.x;
  int nl = 0, nf = 0;
  int types[Q];
  if (cell < n) {
    const int t = flags[cell] & FLAG_TYPE;
    if (t == FLUID && (flags[cell] & FLAG_SLOW)) nl = cell_links<Q>(flags, cell, nx, ny, nz, types);
    nf = (t == INLET || t == OUTLET);
  }
  __shared__ int tl, tf;
  const int pl = block_exclusive_scan(nl, &tl);
  const int pf = block_exclusive_scan(nf, &tf);
  if (nl) {
    long long o = offs[2 * blockIdx.x] + pl;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (types[i]) links[o++] = make_int2((int)cell, i | (types[i] << 8));
  }
  if (nf) fix[offs[2 * blockIdx.x + 1] + pf] = (int)cell;
}

long long bnd_list_blocks(long long n) { return (n + LIST_BLOCK - 1) / LIST_BLOCK; }

int launch_bnd_count(int Q, const uint8_t* flags, int nx, int ny, int nz, int* counts, void* stream) {
  const long long n = (long long)nx * ny * nz;
  const long long b = bnd_list_blocks(n);
  cudaStream_t s = (cudaStream_t)stream;
  if (b > 0x7fffffffLL) return -1;
  if (Q == 9)
    k_bnd_count<9><<<(unsigned)b, LIST_BLOCK, 0, s>>>(flags, n, nx, ny, nz, counts);
  else if (Q == 19)
    k_bnd_count<19><<<(unsigned)b, LIST_BLOCK, 0, s>>>(flags, n, nx, ny, nz, counts);
  else
    k_bnd_count<27><<<(unsigned)b, LIST_BLOCK, 0, s>>>(flags, n, nx, ny, nz, counts);
  return 0;
}

int launch_bnd_write(int Q, const uint8_t* flags, int nx, int ny, int nz, const long long* offs, int2* links,
                     int* fix, void* stream) {
  const long long n = (long long)nx * ny * nz;
  const long long b = bnd_list_blocks(n);
  cudaStream_t s = (cudaStream_t)stream;
  if (b > 0x7fffffffLL) return -1;
  if (Q == 9)
    k_bnd_write<9><<<(unsigned)b, LIST_BLOCK, 0, s>>>(flags, n, nx, ny, nz, offs, links, fix);
  else if (Q == 19)
    k_bnd_write<19><<<(unsigned)b, LIST_BLOCK, 0, s>>>(flags, n, nx, ny, nz, offs, links, fix);
  else
    k_bnd_write<27><<<(unsigned)b, LIST_BLOCK, 0, s>>>(flags, n, nx, ny, nz, offs, links, fix);
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
