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

// Coordinates of a cell index; 32-bit divisions where the lattice allows.
__device__ __forceinline__ void cell_xyz(long long cell, int nx, int ny, bool small, int& x, int& y, int& z) {
  if (small) {
    const unsigned c = (unsigned)cell, r = c / (unsigned)nx;
    x = (int)(c - r * (unsigned)nx);
    y = (int)(r % (unsigned)ny);
    z = (int)(r / (unsigned)ny);
  } else {
    const long long r = cell / nx;
    x = (int)(cell - r * nx);
    y = (int)(r % ny);
    z = (int)(r / ny);
  }
}

// flags = type | FLAG_SLOW where a fluid-like cell has a WALL / LID / EQ cell
// in its Q-stencil, or is an INLET / OUTLET / FWALL cell.  Codes >= 7 set
// err[0]; an INLET, OUTLET or FWALL cell anywhere sets err[2].
template <int Q>
__global__ void k_mask_prepare(const uint8_t* __restrict__ mask, uint8_t* __restrict__ flags, int nx, int ny,
                               int nz, int* err) {
  const long long n = (long long)nx * ny * nz;
  const bool small = n < 0x7fffffffLL;
  bool io = false;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n;
       cell += (long long)gridDim.x * blockDim.x) {
    const int t = mask[cell];
    if (t > FWALL) {
      atomicExch(err, 1);
      flags[cell] = WALL;
      continue;
    }
    int slow = (t == INLET || t == OUTLET || t == FWALL);
    io |= slow != 0;
    if (fluid_like(t) && !slow) {
      int x, y, z;
      cell_xyz(cell, nx, ny, small, x, y, z);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        int xs = x - Lattice<Q>::c(i, 0), ys = y - Lattice<Q>::c(i, 1), zs = z - Lattice<Q>::c(i, 2);
        xs = xs < 0 ? nx - 1 : (xs >= nx ? 0 : xs);
        ys = ys < 0 ? ny - 1 : (ys >= ny ? 0 : ys);
        zs = zs < 0 ? nz - 1 : (zs >= nz ? 0 : zs);
        const int ts = mask[xs + (long long)nx * (ys + (long long)ny * zs)];
        if (!holds_state(ts)) slow = 1;
      }
    }
    flags[cell] = (uint8_t)(t | (slow ? FLAG_SLOW : 0));
  }
  if (io) atomicOr(err + 2, 1);
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

// Boundary tables, built once per mask by compaction in two passes per
// table (per-block counts; an exclusive scan of the counts on the host; then
// ordered per-block writes):
//  - links, direction-major: for each direction i in turn, every FLUID cell,
//    every FWALL cell on an FWALL face plane and every inlet / outlet cell the
//    bulk pass serves, x (ascending), whose source x - c_i is WALL, LID or EQ
//    and not on a face plane, as {x, i | type << 8}.  Consecutive entries
//    then touch consecutive cells of one population plane wherever the wall
//    is not normal to x;
//  - fix-up cells: every other INLET and OUTLET cell and every FWALL cell off
//    the face planes, ascending.
constexpr int LIST_BLOCK = 256;

struct Pred {
  int mode;        // 0: link in direction (cx, cy, cz); 1: fix-up cell
  int cx, cy, cz;  // velocity of the link direction
  int face[6];     // described boundary faces: their sources need no ghost
  int x_in, x_out; // INLET cells of x = 0 / OUTLET cells of x = nx - 1 served by the bulk pass
};

// Does (x, y, z) lie on one of the described face planes?
__device__ __forceinline__ bool on_face_plane(int x, int y, int z, int nx, int ny, int nz, const Pred& pr) {
  return (x == 0 && pr.face[0]) || (x == nx - 1 && pr.face[1]) || (y == 0 && pr.face[2]) ||
         (y == ny - 1 && pr.face[3]) || (nz > 1 && z == 0 && pr.face[4]) || (nz > 1 && z == nz - 1 && pr.face[5]);
}

__device__ __forceinline__ int pred_eval(const uint8_t* __restrict__ flags, long long cell, int nx, int ny, int nz,
                                         const Pred& pr, int* type) {
  const int fl = flags[cell];
  const int t = fl & FLAG_TYPE;
  if (!(t == FLUID || t == FWALL || t == INLET || t == OUTLET)) return 0;
  if (pr.mode == 1 && t == FLUID) return 0;
  if (!(fl & FLAG_SLOW)) return 0;  // a FLUID cell with no WALL / LID / EQ source
  int x, y, z;
  cell_xyz(cell, nx, ny, (long long)nx * ny * nz < 0x7fffffffLL, x, y, z);
  // inlet / outlet cells on the x-planes the bulk pass serves
  const bool io_bulk = (t == INLET && pr.x_in && x == 0) || (t == OUTLET && pr.x_out && x == nx - 1);
  if (pr.mode == 0 && (t == INLET || t == OUTLET) && !io_bulk) return 0;
  // an FWALL cell on a face plane is updated by the bulk pass (it lies on an
  // FWALL face: the host keeps a face only where its plane's cells have the
  // type the faces derive); any other FWALL cell is a fix-up cell
  const bool fw_face = t == FWALL && on_face_plane(x, y, z, nx, ny, nz, pr);
  if (pr.mode == 1) return ((t == INLET || t == OUTLET) && !io_bulk) || (t == FWALL && !fw_face);
  if (t == FWALL && !fw_face) return 0;
  int xs = x - pr.cx, ys = y - pr.cy, zs = z - pr.cz;
  xs = xs < 0 ? nx - 1 : (xs >= nx ? 0 : xs);
  ys = ys < 0 ? ny - 1 : (ys >= ny ? 0 : ys);
  zs = zs < 0 ? nz - 1 : (zs >= nz ? 0 : zs);
  const int ts = flags[xs + (long long)nx * (ys + (long long)ny * zs)] & FLAG_TYPE;
  *type = ts;
  return !holds_state(ts) && !on_face_plane(xs, ys, zs, nx, ny, nz, pr);
}

__global__ void k_pred_count(const uint8_t* __restrict__ flags, long long n, int nx, int ny, int nz, Pred pr,
                             int* counts) {
  const long long cell = blockIdx.x * (long long)LIST_BLOCK + threadIdx.x;
  int t = 0;
  const int hit = cell < n ? pred_eval(flags, cell, nx, ny, nz, pr, &t) : 0;
  const int c = __syncthreads_count(hit);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void k_pred_write(const uint8_t* __restrict__ flags, long long n, int nx, int ny, int nz, Pred pr,
                             int dir, const long long* __restrict__ offs, int2* links, int* cells) {
  __shared__ int warp_base[LIST_BLOCK / 32];
  const long long cell = blockIdx.x * (long long)LIST_BLOCK + threadIdx.x;
  int t = 0;
  const int hit = cell < n ? pred_eval(flags, cell, nx, ny, nz, pr, &t) : 0;
  const unsigned ballot = __ballot_sync(0xffffffffu, hit);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_base[warp] = __popc(ballot);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < LIST_BLOCK / 32; ++w) {
      const int c = warp_base[w];
      warp_base[w] = run;
      run += c;
    }
  }
  __syncthreads();
  if (hit) {
    const long long o = offs[blockIdx.x] + warp_base[warp] + __popc(ballot & ((1u << lane) - 1u));
    if (pr.mode == 1)
      cells[o] = (int)cell;
    else
      links[o] = make_int2((int)cell, dir | (t << 8));
  }
}

long long bnd_list_blocks(long long n) { return (n + LIST_BLOCK - 1) / LIST_BLOCK; }

static Pred make_pred(int mode, int dir, int Q, const int* face, bool x_in, bool x_out) {
  Pred pr;
  pr.mode = mode;
  pr.x_in = x_in ? 1 : 0;
  pr.x_out = x_out ? 1 : 0;
  pr.cx = pr.cy = pr.cz = 0;
  for (int f = 0; f < 6; ++f) pr.face[f] = face ? face[f] : 0;
  if (mode == 0) {
    if (Q == 9) {
      pr.cx = Lattice<9>::c(dir, 0);
      pr.cy = Lattice<9>::c(dir, 1);
    }
    if (Q == 19) {
      pr.cx = Lattice<19>::c(dir, 0);
      pr.cy = Lattice<19>::c(dir, 1);
      pr.cz = Lattice<19>::c(dir, 2);
    }
    if (Q == 27) {
      pr.cx = Lattice<27>::c(dir, 0);
      pr.cy = Lattice<27>::c(dir, 1);
      pr.cz = Lattice<27>::c(dir, 2);
    }
  }
  return pr;
}

int launch_pred_count(int mode, int dir, int Q, const int* face, bool x_in, bool x_out, const uint8_t* flags, int nx,
                      int ny, int nz, int* counts, void* stream) {
  const long long n = (long long)nx * ny * nz;
  const long long b = bnd_list_blocks(n);
  if (b > 0x7fffffffLL) return -1;
  const Pred pr = make_pred(mode, dir, Q, face, x_in, x_out);
  k_pred_count<<<(unsigned)b, LIST_BLOCK, 0, (cudaStream_t)stream>>>(flags, n, nx, ny, nz, pr, counts);
  return 0;
}

int launch_pred_write(int mode, int dir, int Q, const int* face, bool x_in, bool x_out, const uint8_t* flags, int nx,
                      int ny, int nz, const long long* offs, int2* links, int* cells, void* stream) {
  const long long n = (long long)nx * ny * nz;
  const long long b = bnd_list_blocks(n);
  if (b > 0x7fffffffLL) return -1;
  const Pred pr = make_pred(mode, dir, Q, face, x_in, x_out);
  k_pred_write<<<(unsigned)b, LIST_BLOCK, 0, (cudaStream_t)stream>>>(flags, n, nx, ny, nz, pr, dir, offs, links,
                                                                     cells);
  return 0;
}

template <int Q>
__global__ void k_link_cells(const int2* __restrict__ links, long long n, const uint8_t* __restrict__ flags,
                             int nx, int ny, int nz, int2* __restrict__ cells) {
  const bool small = (long long)nx * ny * nz < 0x7fffffffLL;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
    const int2 l = links[e];
    const int i = l.y & 0xff;
    int cx = 0, cy = 0, cz = 0;
#pragma unroll
    for (int j = 1; j < Q; ++j)
      if (j == i) {
        cx = Lattice<Q>::c(j, 0);
        cy = Lattice<Q>::c(j, 1);
        cz = Lattice<Q>::c(j, 2);
      }
    int x, y, z;
    cell_xyz(l.x, nx, ny, small, x, y, z);
    auto wrap = [](int v, int m) { return v < 0 ? m - 1 : (v >= m ? 0 : v); };
    const int w = wrap(x - cx, nx) + nx * (wrap(y - cy, ny) + ny * wrap(z - cz, nz));
    const int b = wrap(x + cx, nx) + nx * (wrap(y + cy, ny) + ny * wrap(z + cz, nz));
    cells[e] = make_int2(w, (flags[b] & FLAG_TYPE) == FLUID ? b : -1);
  }
}

int launch_link_cells(int Q, const int2* links, long long n, const uint8_t* flags, int nx, int ny, int nz,
                      int2* cells, void* stream) {
  if (n <= 0) return 0;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  cudaStream_t s = (cudaStream_t)stream;
  if (Q == 9)
    k_link_cells<9><<<(unsigned)blocks, 256, 0, s>>>(links, n, flags, nx, ny, nz, cells);
  else if (Q == 19)
    k_link_cells<19><<<(unsigned)blocks, 256, 0, s>>>(links, n, flags, nx, ny, nz, cells);
  else if (Q == 27)
    k_link_cells<27><<<(unsigned)blocks, 256, 0, s>>>(links, n, flags, nx, ny, nz, cells);
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

// FP64 sum of squares of n floats (the gradient norm of the differentiable
// workloads); grid-stride, one row (sum, 0, 0, 0) per block.
__global__ void k_sum_squares_partial(const float* __restrict__ x, long long n, double* partial) {
  double acc = 0.0;
  for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256) {
    const double v = x[k];
    acc += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[q];
    partial[4 * (long long)blockIdx.x] = s;
    partial[4 * (long long)blockIdx.x + 1] = 0.0;
    partial[4 * (long long)blockIdx.x + 2] = 0.0;
    partial[4 * (long long)blockIdx.x + 3] = 0.0;
  }
}

long long launch_sum_squares(const float* x, long long n, double* partial, long long capacity, void* stream) {
  long long b = (n + 2047) / 2048;
  if (b > capacity) b = capacity;
  if (b > 65535) b = 65535;
  if (b < 1) b = 1;
  k_sum_squares_partial<<<(unsigned)b, 256, 0, (cudaStream_t)stream>>>(x, n, partial);
  return b;
}

int launch_reduce_final(const double* partial, long long n, double* out, void* stream) {
  k_reduce_final<<<1, 256, 0, (cudaStream_t)stream>>>(partial, n, out);
  return 0;
}

}  // namespace xlb
