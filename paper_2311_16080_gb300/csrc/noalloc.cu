// Allocation-free variant of the FP64 mass / momentum reduction.
//
// Who needs it: callers that cannot call cudaMalloc.  A latency-critical
// loop cannot afford it, because the allocator may synchronise the device and
// takes unbounded time.  A host framework that owns all device memory through
// its own pool allocator, under a fixed memory budget, forbids allocations
// made behind its back.  A recovery path that runs after the device has
// already run out of memory still needs the totals to report the state.
// xlb_reduce keeps its block partial sums in a buffer that each simulation
// context allocates; this entry point instead keeps them in one fixed array
// compiled into the library, so a call touches only memory that already
// exists.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (128 KiB) until the process exits.  All calls on a device
// share it, so calls whose kernels overlap on the GPU (different streams, or
// different host threads without ordering) race on it; order them on one
// stream.  Each call writes every partial row it reads, so nothing has to be
// cleared between calls.
//
// The call sums the populations as they are stored.  After xlb_step the live
// buffer of a simulation holds the post-collision state h_{t-1} (the pull of
// the next update streams it), not the post-stream state f_t that
// xlb_reduce sums; on a periodic lattice without a body force the totals of
// the two agree (collision and streaming conserve mass and momentum), on a
// lattice with walls, inlets or a moving lid they differ.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/xlb.h"
#include "lattice.cuh"
#include "xlb_types.h"

namespace xlb {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 64;
constexpr long long NA_CELLS_PER_BLOCK = (long long)NA_THREADS * NA_CELLS_PER_THREAD;  // 16384
constexpr int NA_MAX_PARTIALS = 4096;  // 4096 rows x 4 doubles = 128 KiB
constexpr long long NA_MAX_CELLS = NA_CELLS_PER_BLOCK * NA_MAX_PARTIALS;  // 67,108,864

// The fixed scratch: one row (mass, j_x, j_y, j_z) per block, then the result.
static __device__ __align__(256) double g_noalloc_scratch[4 * NA_MAX_PARTIALS + 4];

// Block b sums the FP64 moments of cells [b * 16384, (b + 1) * 16384) of the
// stored populations (deviations df_i = f_i - w_i, read in place) over the
// fluid-like cells of `mask` (all cells if mask is null).
template <int Q, typename S>
__global__ void __launch_bounds__(NA_THREADS) k_moments_partial_static(const S* __restrict__ f, long long plane,
                                                                       long long n, const uint8_t* __restrict__ mask,
                                                                       double* partial) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int k = 0; k < NA_CELLS_PER_THREAD; ++k) {
    const long long cell = base + (long long)k * NA_THREADS + threadIdx.x;
    if (cell >= n) break;
    if (mask && !fluid_like(mask[cell])) continue;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double fi = weight_d<Q>(i) + (double)Store<S>::ld(f + (long long)i * plane + cell);
      acc[0] += fi;
      acc[1] += Lattice<Q>::c(i, 0) * fi;
      acc[2] += Lattice<Q>::c(i, 1) * fi;
      acc[3] += Lattice<Q>::c(i, 2) * fi;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  __shared__ double red[NA_THREADS / 32][4];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[threadIdx.x >> 5][k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int w = 0; w < NA_THREADS / 32; ++w) s += red[w][k];
      partial[4 * (long long)blockIdx.x + k] = s;
    }
}

// Fixed-order sum of the nb partial rows into out[0..3].
__global__ void k_moments_final_static(const double* __restrict__ partial, int nb, double* out) {
  __shared__ double s[4][NA_THREADS];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = threadIdx.x; r < nb; r += NA_THREADS)
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] += partial[4 * r + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 4; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

template <int Q, typename S>
void launch_partial(const void* f, long long plane, long long n, const uint8_t* mask, double* partial, int nb,
                    cudaStream_t st) {
  k_moments_partial_static<Q, S><<<nb, NA_THREADS, 0, st>>>((const S*)f, plane, n, mask, partial);
}

// Device address of the scratch array, looked up once per device.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {};

}  // namespace
}  // namespace xlb

using namespace xlb;

extern "C" int xlb_moments_noalloc(int lattice, const int64_t dims[3], int storage, const void* populations,
                                   int64_t plane_stride, const uint8_t* mask, double* out, void* cuda_stream) {
  if (lattice != 9 && lattice != 19 && lattice != 27) return XLB_ERR_ARG;
  if (!dims || !populations || !out) return XLB_ERR_ARG;
  if (storage < XLB_STORE_F32 || storage > XLB_STORE_BF16) return XLB_ERR_ARG;
  const long long nx = dims[0], ny = dims[1], nz = dims[2];
  if (nx < 1 || ny < 1 || nz < 1 || (lattice == 9 && nz != 1)) return XLB_ERR_ARG;
  // the fixed scratch holds 4096 partial rows of 16384 cells each; the
  // product is checked factor by factor so that it cannot overflow
  if (nx > NA_MAX_CELLS || ny > NA_MAX_CELLS / nx || nz > NA_MAX_CELLS / (nx * ny)) return XLB_ERR_ARG;
  const long long n = nx * ny * nz;
  if (plane_stride < n) return XLB_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return XLB_ERR_CUDA;
  double* scratch = nullptr;
  {
    // first call on this device: find the array's device address (with this
    // device current); later calls reuse it
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return XLB_ERR_CUDA;
      }
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  cudaPointerAttributes attr;
  bool out_on_device = false;
  if (cudaPointerGetAttributes(&attr, out) == cudaSuccess)
    out_on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
  else
    cudaGetLastError();
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!out_on_device) {
    // a host result needs a copy and a synchronisation of the stream, which
    // a stream that is being captured does not allow
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
      cudaGetLastError();
      return XLB_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return XLB_ERR_ARG;
  }
  const int nb = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  double* result = scratch + 4 * NA_MAX_PARTIALS;
  const int Q = lattice;
  if (Q == 9) {
    if (storage == XLB_STORE_F32) launch_partial<9, float>(populations, plane_stride, n, mask, scratch, nb, st);
    if (storage == XLB_STORE_F16) launch_partial<9, __half>(populations, plane_stride, n, mask, scratch, nb, st);
    if (storage == XLB_STORE_BF16)
      launch_partial<9, __nv_bfloat16>(populations, plane_stride, n, mask, scratch, nb, st);
  } else if (Q == 19) {
    if (storage == XLB_STORE_F32) launch_partial<19, float>(populations, plane_stride, n, mask, scratch, nb, st);
    if (storage == XLB_STORE_F16) launch_partial<19, __half>(populations, plane_stride, n, mask, scratch, nb, st);
    if (storage == XLB_STORE_BF16)
      launch_partial<19, __nv_bfloat16>(populations, plane_stride, n, mask, scratch, nb, st);
  } else {
    if (storage == XLB_STORE_F32) launch_partial<27, float>(populations, plane_stride, n, mask, scratch, nb, st);
    if (storage == XLB_STORE_F16) launch_partial<27, __half>(populations, plane_stride, n, mask, scratch, nb, st);
    if (storage == XLB_STORE_BF16)
      launch_partial<27, __nv_bfloat16>(populations, plane_stride, n, mask, scratch, nb, st);
  }
  k_moments_final_static<<<1, NA_THREADS, 0, st>>>(scratch, nb, out_on_device ? out : result);
  if (cudaGetLastError() != cudaSuccess) return XLB_ERR_CUDA;
  if (!out_on_device) {
    if (cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return XLB_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return XLB_ERR_CUDA;
  }
  return XLB_OK;
}
