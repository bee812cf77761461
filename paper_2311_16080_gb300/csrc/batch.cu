// Batched small 2D domains (the batching of Section 6: many independent
// simulations advanced together).  Thousands of D2Q9 domains of different
// sizes, each periodic in x and y unless its mask says otherwise, with WALL
// cells (halfway bounce-back) and a per-domain body force, advance in one
// persistent launch: every CTA takes domains from an atomic queue (largest
// first) and runs all requested steps of a domain before taking the next,
// with a CTA barrier between steps.  A domain's state therefore stays in the
// caches of one SM while it is being advanced.  The launch and its queue
// reset are captured in a CUDA graph and replayed.
//
// Per domain: populations f[i][y][x] (deviations f_i - w_i, like the single
// lattice) in two buffers, a flag byte per cell (type | FLAG_SLOW when a WALL
// cell is in the 3x3 stencil).
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/xlb.h"
#include "lbm_device.cuh"

namespace xlb {
namespace {

struct BatchDom {
  long long off;   // element offset of the domain's populations in each buffer
  long long foff;  // offset of its flag bytes
  int nx, ny;
  int plane;       // elements between population planes (nx * ny rounded up to 64)
  float Fx, Fy;
};

// One update of every cell of one domain: pull with periodic wrap and
// halfway bounce-back from WALL sources, BGK + exact-difference force, store.
template <typename S>
__device__ __forceinline__ void batch_domain_step(const S* __restrict__ src, S* __restrict__ dst,
                                                  const uint8_t* __restrict__ fl, const BatchDom& d, float omega) {
  const int n = d.nx * d.ny;
  StepParams p;
  p.omega = omega;
  p.has_force = (d.Fx != 0.f || d.Fy != 0.f);
  p.F[0] = d.Fx;
  p.F[1] = d.Fy;
  p.F[2] = 0.f;
  for (int cell = threadIdx.x; cell < n; cell += blockDim.x) {
    const int x = cell % d.nx, y = cell / d.nx;
    const int f = __ldg(fl + cell);
    const int xm = x == 0 ? d.nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
    const int xs[3] = {xm, x, xp}, rows[3] = {ym * d.nx, y * d.nx, yp * d.nx};
    float df[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int s = xs[1 - Lattice<9>::c(i, 0)] + rows[1 - Lattice<9>::c(i, 1)];
      df[i] = Store<S>::ld_l2(src + (long long)i * d.plane + s);
    }
    if (f & FLAG_SLOW) {
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int s = xs[1 - Lattice<9>::c(i, 0)] + rows[1 - Lattice<9>::c(i, 1)];
        if ((__ldg(fl + s) & FLAG_TYPE) == WALL) df[i] = Store<S>::ld_l2(src + (long long)opposite<9>(i) * d.plane + cell);
      }
    }
    collide<9, COLL_BGK>(df, p);
    if ((f & FLAG_TYPE) == FLUID) {
      CellRound<S> rnd;
      rnd.begin((uint32_t)(d.off + cell), df);
#pragma unroll
      for (int i = 0; i < 9; ++i) rnd.st_l2(dst + (long long)i * d.plane + cell, i, df[i]);
    }
  }
}

// Persistent launch: domains from the queue, `steps` updates each.
// Buffers: after an even number of steps the state is back in A.
template <typename S>
__global__ void k_batch_persistent(const BatchDom* __restrict__ doms, const int* __restrict__ order, int n_dom,
                                   S* A, S* B, const uint8_t* __restrict__ flags, float omega, int steps,
                                   int* counter) {
  __shared__ int s_q;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(counter, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();  // every thread has read s_q before it is overwritten
    if (q >= n_dom) return;
    const BatchDom d = doms[order[q]];
    S* a = A + d.off;
    S* b = B + d.off;
    const uint8_t* fl = flags + d.foff;
    for (int t = 0; t < steps; ++t) {
      batch_domain_step<S>(a, b, fl, d, omega);
      __syncthreads();  // the whole domain is updated before the next step reads it
      S* tmp = a;
      a = b;
      b = tmp;
    }
  }
}

// One step of one domain with an ordinary grid (the launch-per-domain
// baseline): block b updates cells [b * blockDim, (b + 1) * blockDim).
template <typename S>
__global__ void k_batch_single(const BatchDom* __restrict__ doms, int dom, const S* A, S* B,
                               const uint8_t* __restrict__ flags, float omega) {
  const BatchDom d = doms[dom];
  const int n = d.nx * d.ny;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const S* src = A + d.off;
  S* dst = B + d.off;
  const uint8_t* fl = flags + d.foff;
  StepParams p;
  p.omega = omega;
  p.has_force = (d.Fx != 0.f || d.Fy != 0.f);
  p.F[0] = d.Fx;
  p.F[1] = d.Fy;
  p.F[2] = 0.f;
  const int x = cell % d.nx, y = cell / d.nx;
  const int f = __ldg(fl + cell);
  const int xm = x == 0 ? d.nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
  const int xs[3] = {xm, x, xp}, rows[3] = {ym * d.nx, y * d.nx, yp * d.nx};
  float df[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int s = xs[1 - Lattice<9>::c(i, 0)] + rows[1 - Lattice<9>::c(i, 1)];
    df[i] = Store<S>::ld_l2(src + (long long)i * d.plane + s);
  }
  if (f & FLAG_SLOW) {
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const int s = xs[1 - Lattice<9>::c(i, 0)] + rows[1 - Lattice<9>::c(i, 1)];
      if ((__ldg(fl + s) & FLAG_TYPE) == WALL) df[i] = Store<S>::ld_l2(src + (long long)opposite<9>(i) * d.plane + cell);
    }
  }
  collide<9, COLL_BGK>(df, p);
  if ((f & FLAG_TYPE) == FLUID) {
    CellRound<S> rnd;
    rnd.begin((uint32_t)(d.off + cell), df);
#pragma unroll
    for (int i = 0; i < 9; ++i) rnd.st_l2(dst + (long long)i * d.plane + cell, i, df[i]);
  }
}

// f_0 = f^eq(rho, u) per cell (all domains in one launch over the
// concatenated fields; a binary search of cell_start finds the domain).
template <typename S>
__global__ void k_batch_init(const BatchDom* __restrict__ doms, const int* __restrict__ cell_start, int n_dom,
                             long long total, S* A, const float* rho, const float* u, const uint8_t* flags) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n_dom - 1;
  while (lo < hi) {  // last domain whose first cell is <= g
    const int mid = (lo + hi + 1) / 2;
    if (cell_start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const BatchDom d = doms[lo];
  const int cell = (int)(g - cell_start[lo]);
  const float r = rho ? rho[g] : 1.0f;
  float v[3] = {u ? u[2 * g] : 0.f, u ? u[2 * g + 1] : 0.f, 0.f};
  const bool fluid = (flags[d.foff + cell] & FLAG_TYPE) == FLUID;
  const float usq = v[0] * v[0] + v[1] * v[1];
  float df[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) df[i] = fluid ? weight<9>(i) * ((r - 1.0f) + r * eq_poly<9>(i, v, usq)) : 0.f;
  CellRound<S> rnd;
  rnd.begin((uint32_t)(d.off + cell), df);
#pragma unroll
  for (int i = 0; i < 9; ++i) rnd.st(A + d.off + (long long)i * d.plane + cell, i, df[i]);
}

// rho and reported u = (j + F/2) / rho per cell (0 on WALL cells), from the
// stored post-collision state: the pull is applied as in an update.
template <typename S>
__global__ void k_batch_macro(const BatchDom* __restrict__ doms, const int* __restrict__ cell_start, int n_dom,
                              long long total, const S* A, const uint8_t* flags, int kind_h, float* rho, float* u) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n_dom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (cell_start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const BatchDom d = doms[lo];
  const int cell = (int)(g - cell_start[lo]);
  const uint8_t* fl = flags + d.foff;
  const S* src = A + d.off;
  const int f = fl[cell];
  float r = 0.f, ux = 0.f, uy = 0.f;
  if ((f & FLAG_TYPE) == FLUID) {
    const int x = cell % d.nx, y = cell / d.nx;
    const int xm = x == 0 ? d.nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
    const int xs[3] = {xm, x, xp}, rows[3] = {ym * d.nx, y * d.nx, yp * d.nx};
    float df[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int s = kind_h ? xs[1 - Lattice<9>::c(i, 0)] + rows[1 - Lattice<9>::c(i, 1)] : cell;
      float v = Store<S>::ld(src + (long long)i * d.plane + s);
      if (kind_h && (fl[s] & FLAG_TYPE) == WALL) v = Store<S>::ld(src + (long long)opposite<9>(i) * d.plane + cell);
      df[i] = v;
    }
    float drho, j[3];
    moments<9>(df, drho, j);
    r = 1.0f + drho;
    ux = (j[0] + 0.5f * d.Fx) / r;
    uy = (j[1] + 0.5f * d.Fy) / r;
  }
  if (rho) rho[g] = r;
  if (u) {
    u[2 * g] = ux;
    u[2 * g + 1] = uy;
  }
}

// Local collision of the initial state (the first update after init).
template <typename S>
__global__ void k_batch_collide(const BatchDom* __restrict__ doms, const int* __restrict__ cell_start, int n_dom,
                                long long total, S* A, const uint8_t* flags, float omega) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n_dom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (cell_start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const BatchDom d = doms[lo];
  const int cell = (int)(g - cell_start[lo]);
  if ((flags[d.foff + cell] & FLAG_TYPE) != FLUID) return;
  StepParams p;
  p.omega = omega;
  p.has_force = (d.Fx != 0.f || d.Fy != 0.f);
  p.F[0] = d.Fx;
  p.F[1] = d.Fy;
  p.F[2] = 0.f;
  float df[9];
  S* a = A + d.off + cell;
#pragma unroll
  for (int i = 0; i < 9; ++i) df[i] = Store<S>::ld_plain(a + (long long)i * d.plane);
  collide<9, COLL_BGK>(df, p);
  CellRound<S> rnd;
  rnd.begin((uint32_t)(d.off + cell), df);
#pragma unroll
  for (int i = 0; i < 9; ++i) rnd.st(a + (long long)i * d.plane, i, df[i]);
}

// Flags: type | FLAG_SLOW for FLUID cells with a WALL cell in the stencil;
// codes other than FLUID / WALL set *err.
__global__ void k_batch_flags(const BatchDom* __restrict__ doms, const int* __restrict__ cell_start, int n_dom,
                              long long total, const uint8_t* mask_cat, uint8_t* flags, int* err) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n_dom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (cell_start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const BatchDom d = doms[lo];
  const int cell = (int)(g - cell_start[lo]);
  const uint8_t* m = mask_cat + cell_start[lo];
  const int t = m[cell];
  if (t != FLUID && t != WALL) {
    atomicExch(err, 1);
    flags[d.foff + cell] = WALL;
    return;
  }
  int slow = 0;
  if (t == FLUID) {
    const int x = cell % d.nx, y = cell / d.nx;
    for (int i = 1; i < 9; ++i) {
      int xs = x - Lattice<9>::c(i, 0), ys = y - Lattice<9>::c(i, 1);
      xs = xs < 0 ? d.nx - 1 : (xs >= d.nx ? 0 : xs);
      ys = ys < 0 ? d.ny - 1 : (ys >= d.ny ? 0 : ys);
      if (m[xs + d.nx * ys] == WALL) slow = 1;
    }
  }
  flags[d.foff + cell] = (uint8_t)(t | (slow ? FLAG_SLOW : 0));
}

}  // namespace
}  // namespace xlb

using namespace xlb;

struct xlb_batch {
  int n = 0, storage = 0, esize = 4;
  double omega = 1.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<BatchDom> hdoms;
  std::vector<int> hstart;  // first concatenated cell of each domain (+ total)
  long long total_cells = 0, total_elems = 0, total_flags = 0;
  BatchDom* doms = nullptr;
  int* order = nullptr;
  int* start = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  int kind_h = 0;
  int64_t t = 0;
  uint8_t* flags = nullptr;
  bool has_mask = false;
  int* counter = nullptr;  // [0] queue, [1] error word
  int threads = 256, ctas_per_sm = 2, num_sms = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_steps = -1, graph_threads = 0, graph_grid = 0, graph_cur = -1;
  std::string err;
};

static int bfail(xlb_batch* b, int code, const char* msg) {
  if (b) b->err = msg;
  return code;
}

#define BCK(call)                                                      \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      if (b) b->err = std::string(#call ": ") + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? XLB_ERR_OOM : XLB_ERR_CUDA; \
    }                                                                  \
  } while (0)

template <typename F>
static void by_storage(int storage, F&& f) {
  if (storage == XLB_STORE_F32) f(float());
  if (storage == XLB_STORE_F16) f(__half());
  if (storage == XLB_STORE_BF16) f(__nv_bfloat16());
}

static unsigned grid_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }

extern "C" {

void xlb_batch_destroy(xlb_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int k = 0; k < 2; ++k)
    if (b->buf[k]) cudaFree(b->buf[k]);
  if (b->doms) cudaFree(b->doms);
  if (b->order) cudaFree(b->order);
  if (b->start) cudaFree(b->start);
  if (b->flags) cudaFree(b->flags);
  if (b->counter) cudaFree(b->counter);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* xlb_batch_last_error(const xlb_batch* b) { return b ? b->err.c_str() : ""; }

int xlb_batch_create(xlb_batch** out, int n_domains, const int32_t* nx, const int32_t* ny, double omega,
                     int storage, void* cuda_stream) {
  if (!out) return XLB_ERR_ARG;
  *out = nullptr;
  if (n_domains < 1 || !nx || !ny) return XLB_ERR_ARG;
  if (!(omega > 0.0 && omega < 2.0)) return XLB_ERR_ARG;
  if (storage < XLB_STORE_F32 || storage > XLB_STORE_BF16) return XLB_ERR_ARG;
  xlb_batch* b = new xlb_batch();
  b->n = n_domains;
  b->storage = storage;
  b->esize = storage == XLB_STORE_F32 ? 4 : 2;
  b->omega = omega;
  long long off = 0, foff = 0, cells = 0;
  for (int d = 0; d < n_domains; ++d) {
    if (nx[d] < 1 || ny[d] < 1 || (long long)nx[d] * ny[d] > (1LL << 26)) {
      delete b;
      return XLB_ERR_ARG;
    }
    BatchDom bd;
    bd.nx = nx[d];
    bd.ny = ny[d];
    bd.plane = (nx[d] * ny[d] + 63) / 64 * 64;
    bd.off = off;
    bd.foff = foff;
    bd.Fx = bd.Fy = 0.f;
    b->hdoms.push_back(bd);
    b->hstart.push_back((int)cells);
    off += 9LL * bd.plane;
    foff += (long long)nx[d] * ny[d];
    cells += (long long)nx[d] * ny[d];
  }
  if (cells > 0x7fffffffLL) {
    delete b;
    return XLB_ERR_UNSUPPORTED;
  }
  b->hstart.push_back((int)cells);
  b->total_cells = cells;
  b->total_elems = off;
  b->total_flags = foff;
  auto bail = [&](int code) {
    xlb_batch_destroy(b);
    return code;
  };
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(XLB_ERR_CUDA);
    b->own_stream = true;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bail(XLB_ERR_CUDA);
  for (int k = 0; k < 2; ++k)
    if (cudaMalloc(&b->buf[k], b->esize * (size_t)off) != cudaSuccess) return bail(XLB_ERR_OOM);
  if (cudaMalloc(&b->doms, sizeof(BatchDom) * n_domains) != cudaSuccess ||
      cudaMalloc(&b->order, sizeof(int) * n_domains) != cudaSuccess ||
      cudaMalloc(&b->start, sizeof(int) * (n_domains + 1)) != cudaSuccess ||
      cudaMalloc(&b->flags, (size_t)foff) != cudaSuccess || cudaMalloc(&b->counter, 4 * sizeof(int)) != cudaSuccess)
    return bail(XLB_ERR_OOM);
  // queue order: largest domain first (longest-processing-time first)
  std::vector<int> ord(n_domains);
  for (int d = 0; d < n_domains; ++d) ord[d] = d;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) {
    return (long long)nx[a] * ny[a] > (long long)nx[c] * ny[c];
  });
  if (cudaMemcpy(b->doms, b->hdoms.data(), sizeof(BatchDom) * n_domains, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->order, ord.data(), sizeof(int) * n_domains, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->start, b->hstart.data(), sizeof(int) * (n_domains + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->counter, 0, 4 * sizeof(int)) != cudaSuccess || cudaMemset(b->flags, 0, (size_t)foff) != cudaSuccess)
    return bail(XLB_ERR_CUDA);
  *out = b;
  return XLB_OK;
}

int xlb_batch_set_masks(xlb_batch* b, const uint8_t* masks, const float* forces) {
  if (!b) return XLB_ERR_ARG;
  if (forces) {
    for (int d = 0; d < b->n; ++d) {
      b->hdoms[d].Fx = forces[2 * d];
      b->hdoms[d].Fy = forces[2 * d + 1];
    }
    BCK(cudaMemcpyAsync(b->doms, b->hdoms.data(), sizeof(BatchDom) * b->n, cudaMemcpyHostToDevice, b->stream));
  }
  if (masks) {
    uint8_t* dm = nullptr;
    BCK(cudaMalloc(&dm, (size_t)b->total_cells));
    cudaError_t e = cudaMemcpyAsync(dm, masks, (size_t)b->total_cells, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->counter + 1, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) {
      k_batch_flags<<<grid_of(b->total_cells, 256), 256, 0, b->stream>>>(b->doms, b->start, b->n, b->total_cells, dm,
                                                                         b->flags, b->counter + 1);
      e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, b->counter + 1, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(dm);
    if (e != cudaSuccess) return bfail(b, XLB_ERR_CUDA, cudaGetErrorString(e));
    if (herr) return bfail(b, XLB_ERR_UNSUPPORTED, "batched domains take FLUID and WALL cells only");
    b->has_mask = true;
  }
  return XLB_OK;
}

int xlb_batch_init(xlb_batch* b, const float* rho, const float* u) {
  if (!b) return XLB_ERR_ARG;
  float* dr = nullptr;
  float* du = nullptr;
  const size_t n = (size_t)b->total_cells;
  if (rho) BCK(cudaMalloc(&dr, n * sizeof(float)));
  if (u) BCK(cudaMalloc(&du, 2 * n * sizeof(float)));
  if (rho) BCK(cudaMemcpyAsync(dr, rho, n * sizeof(float), cudaMemcpyDefault, b->stream));
  if (u) BCK(cudaMemcpyAsync(du, u, 2 * n * sizeof(float), cudaMemcpyDefault, b->stream));
  by_storage(b->storage, [&](auto tag) {
    using S = decltype(tag);
    k_batch_init<S><<<grid_of(b->total_cells, 256), 256, 0, b->stream>>>(
        b->doms, b->start, b->n, b->total_cells, (S*)b->buf[0], dr, du, b->flags);
  });
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(b->stream);
  if (dr) cudaFree(dr);
  if (du) cudaFree(du);
  if (e != cudaSuccess) return bfail(b, XLB_ERR_CUDA, cudaGetErrorString(e));
  b->cur = 0;
  b->kind_h = 0;
  b->t = 0;
  return XLB_OK;
}

// First update after init: a local collision.
static int batch_first(xlb_batch* b) {
  by_storage(b->storage, [&](auto tag) {
    using S = decltype(tag);
    k_batch_collide<S><<<grid_of(b->total_cells, 256), 256, 0, b->stream>>>(
        b->doms, b->start, b->n, b->total_cells, (S*)b->buf[b->cur], b->flags, (float)b->omega);
  });
  if (cudaGetLastError() != cudaSuccess) return bfail(b, XLB_ERR_CUDA, "batch collide launch");
  b->kind_h = 1;
  b->t += 1;
  return XLB_OK;
}

int xlb_batch_set_launch(xlb_batch* b, int threads, int ctas_per_sm) {
  if (!b) return XLB_ERR_ARG;
  if (threads < 32 || threads > 1024 || threads % 32 || ctas_per_sm < 1 || ctas_per_sm > 32)
    return bfail(b, XLB_ERR_ARG, "threads must be 32..1024 (multiple of 32), CTAs per SM 1..32");
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  return XLB_OK;
}

int xlb_batch_step(xlb_batch* b, int64_t n) {
  if (!b) return XLB_ERR_ARG;
  if (n < 0 || n > 0x7fffffff) return bfail(b, XLB_ERR_ARG, "n out of range");
  if (!b->has_mask) return bfail(b, XLB_ERR_STATE, "set the domain masks first");
  if (n == 0) return XLB_OK;
  if (!b->kind_h) {
    int r = batch_first(b);
    if (r) return r;
    if (--n == 0) return XLB_OK;
  }
  // resident CTAs of the chosen shape
  int occ = 0;
  by_storage(b->storage, [&](auto tag) {
    using S = decltype(tag);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_persistent<S>, b->threads, 0);
  });
  const int per_sm = std::max(1, std::min(occ, b->ctas_per_sm));
  const int grid = std::min(b->n, per_sm * b->num_sms);
  // (re)build the graph of {queue reset, persistent launch} when its shape changes
  if (!b->graph_exec || b->graph_steps != (int)n || b->graph_threads != b->threads || b->graph_grid != grid ||
      b->graph_cur != b->cur) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream);
    by_storage(b->storage, [&](auto tag) {
      using S = decltype(tag);
      k_batch_persistent<S><<<grid, b->threads, 0, b->stream>>>(b->doms, b->order, b->n, (S*)b->buf[b->cur],
                                                                 (S*)b->buf[b->cur ^ 1], b->flags, (float)b->omega,
                                                                 (int)n, b->counter);
    });
    BCK(cudaStreamEndCapture(b->stream, &b->graph));
    BCK(cudaGraphInstantiate(&b->graph_exec, b->graph, 0));
    b->graph_steps = (int)n;
    b->graph_threads = b->threads;
    b->graph_grid = grid;
    b->graph_cur = b->cur;
  }
  BCK(cudaGraphLaunch(b->graph_exec, b->stream));
  if (n & 1) b->cur ^= 1;
  b->t += n;
  return XLB_OK;
}

int xlb_batch_step_per_domain(xlb_batch* b, int64_t n) {
  if (!b) return XLB_ERR_ARG;
  if (n < 0) return bfail(b, XLB_ERR_ARG, "n out of range");
  if (!b->has_mask) return bfail(b, XLB_ERR_STATE, "set the domain masks first");
  for (int64_t k = 0; k < n; ++k) {
    if (!b->kind_h) {
      int r = batch_first(b);
      if (r) return r;
      continue;
    }
    for (int d = 0; d < b->n; ++d) {
      const long long cells = (long long)b->hdoms[d].nx * b->hdoms[d].ny;
      by_storage(b->storage, [&](auto tag) {
        using S = decltype(tag);
        k_batch_single<S><<<grid_of(cells, 128), 128, 0, b->stream>>>(b->doms, d, (const S*)b->buf[b->cur],
                                                                       (S*)b->buf[b->cur ^ 1], b->flags,
                                                                       (float)b->omega);
      });
    }
    if (cudaGetLastError() != cudaSuccess) return bfail(b, XLB_ERR_CUDA, "per-domain launch");
    b->cur ^= 1;
    b->t += 1;
  }
  return XLB_OK;
}

int xlb_batch_macroscopic(xlb_batch* b, float* rho, float* u) {
  if (!b) return XLB_ERR_ARG;
  const size_t n = (size_t)b->total_cells;
  float* dr = nullptr;
  float* du = nullptr;
  BCK(cudaMalloc(&dr, n * sizeof(float)));
  cudaError_t e = cudaMalloc(&du, 2 * n * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(dr);
    return bfail(b, XLB_ERR_OOM, "readout buffers");
  }
  by_storage(b->storage, [&](auto tag) {
    using S = decltype(tag);
    k_batch_macro<S><<<grid_of(b->total_cells, 256), 256, 0, b->stream>>>(
        b->doms, b->start, b->n, b->total_cells, (const S*)b->buf[b->cur], b->flags, b->kind_h, dr, du);
  });
  e = cudaGetLastError();
  if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, dr, n * sizeof(float), cudaMemcpyDefault, b->stream);
  if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, 2 * n * sizeof(float), cudaMemcpyDefault, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(dr);
  cudaFree(du);
  if (e != cudaSuccess) return bfail(b, XLB_ERR_CUDA, cudaGetErrorString(e));
  return XLB_OK;
}

int xlb_batch_info(const xlb_batch* b, int64_t* total_cells, int64_t* t, int* threads, int* ctas_per_sm) {
  if (!b || !total_cells || !t || !threads || !ctas_per_sm) return XLB_ERR_ARG;
  *total_cells = b->total_cells;
  *t = b->t;
  *threads = b->threads;
  *ctas_per_sm = b->ctas_per_sm;
  return XLB_OK;
}

// Autotuner: times each launch shape (threads per CTA x resident CTAs per SM)
// over `sample_steps` updates on a copy of the state (restored after every
// trial, so tuning does not advance the simulation), keeps the fastest, and
// records it in `cache_path` (one line per batch geometry; a hit skips the
// timing).  cache_path may be NULL.
int xlb_batch_tune(xlb_batch* b, int sample_steps, const char* cache_path, int* best_threads, int* best_ctas) {
  if (!b) return XLB_ERR_ARG;
  if (sample_steps < 2) return bfail(b, XLB_ERR_ARG, "sample_steps must be >= 2");
  if (!b->has_mask) return bfail(b, XLB_ERR_STATE, "set the domain masks first");
  char key[256];
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  snprintf(key, sizeof key, "batch-d2q9 n=%d cells=%lld storage=%d sms=%d %s", b->n, b->total_cells, b->storage,
           b->num_sms, prop.name);
  if (cache_path) {
    FILE* fh = fopen(cache_path, "r");
    if (fh) {
      char line[512];
      while (fgets(line, sizeof line, fh)) {
        char* q = strstr(line, "\"key\": \"");
        if (!q || strncmp(q + 9, key, strlen(key)) != 0 || q[9 + strlen(key)] != '"') continue;
        int th = 0, ct = 0;
        const char* a = strstr(line, "\"threads\": ");
        const char* c = strstr(line, "\"ctas_per_sm\": ");
        if (a && c && sscanf(a + 11, "%d", &th) == 1 && sscanf(c + 15, "%d", &ct) == 1 &&
            xlb_batch_set_launch(b, th, ct) == XLB_OK) {
          fclose(fh);
          if (best_threads) *best_threads = th;
          if (best_ctas) *best_ctas = ct;
          return XLB_OK;
        }
      }
      fclose(fh);
    }
  }
  const size_t bytes = (size_t)b->esize * (size_t)b->total_elems;
  void* save = nullptr;
  BCK(cudaMalloc(&save, bytes));
  const int cur0 = b->cur, kind0 = b->kind_h;
  const int64_t t0 = b->t;
  cudaError_t e = cudaMemcpyAsync(save, b->buf[cur0], bytes, cudaMemcpyDeviceToDevice, b->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cand_t[4] = {128, 256, 512, 1024};
  const int cand_c[4] = {1, 2, 4, 8};
  float best = 1e30f;
  int bt = b->threads, bc = b->ctas_per_sm;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    for (int j = 0; j < 4 && e == cudaSuccess; ++j) {
      if (cand_t[i] * cand_c[j] > 2048) continue;
      xlb_batch_set_launch(b, cand_t[i], cand_c[j]);
      if (!b->kind_h && batch_first(b) != XLB_OK) break;
      cudaEventRecord(e0, b->stream);
      if (xlb_batch_step(b, sample_steps) != XLB_OK) break;
      cudaEventRecord(e1, b->stream);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bt = cand_t[i];
        bc = cand_c[j];
      }
      // restore the state
      b->cur = cur0;
      b->kind_h = kind0;
      b->t = t0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(b->buf[cur0], save, bytes, cudaMemcpyDeviceToDevice, b->stream);
    }
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return bfail(b, XLB_ERR_CUDA, cudaGetErrorString(e));
  xlb_batch_set_launch(b, bt, bc);
  if (best_threads) *best_threads = bt;
  if (best_ctas) *best_ctas = bc;
  if (cache_path) {
    FILE* fh = fopen(cache_path, "a");
    if (fh) {
      fprintf(fh, "{\"key\": \"%s\", \"threads\": %d, \"ctas_per_sm\": %d, \"ms\": %.4f}\n", key, bt, bc, best);
      fclose(fh);
    }
  }
  return XLB_OK;
}

int xlb_batch_synchronize(xlb_batch* b) {
  if (!b) return XLB_ERR_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  return XLB_OK;
}

}  // extern "C"
