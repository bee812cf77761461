// Host implementation of the C ABI declared in include/xlb.h.
//
// State machine of a ctx:
//  - xlb_init writes f_0 (post-stream populations) and marks the buffer as
//    "pre-collision" (kind_h = 0).  The first step after that is a local
//    collision (h_0 = C(f_0)); every later step is one fused stream-collide
//    launch h_t = C(S_bc(h_{t-1})).  The stored buffer after t steps is
//    h_{t-1}, and the observables of f_t = S_bc(h_{t-1}) are computed by a pull
//    inside the readout kernels.  (S_bc C)^n = S_bc (C S_bc)^(n-1) C, so this is
//    the same sequence of operations as Eqs. 1-2 applied n times.
//  - A tape records h_{sk-1} at every time sk < T; the adjoint recomputes one
//    segment of k states from its checkpoint before walking it backwards.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/xlb.h"
#include "adjoint.h"
#include "lattice.cuh"
#include "launch.h"
#include "lattice.cuh"

using namespace xlb;

struct EventPair {
  cudaEvent_t a, b;
};

struct xlb_ctx {
  int Q = 0, D = 0, coll = 0, storage = 0, esize = 4;
  int64_t nx = 0, ny = 0, nz = 0;
  long long N = 0, plane = 0;
  double omega = 1.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  uint8_t* flags = nullptr;
  bool has_mask = false;
  int2* links = nullptr;  // ghost links {cell, dir | type << 8} of the mask
  long long n_links = 0;
  int2* link_cells = nullptr;        // per link: source cell, Bouzidi partner (k_link_cells)
  int* fix = nullptr;  // fix-up cells: inlet / outlet cells off whole x-planes, FWALL cells off the faces
  long long n_fix = 0;
  void* fix_side = nullptr;  // Q x n_fix values of the storage type: their recomputed update
  // auxiliary stream on which the fix-up cells are recomputed beside the bulk
  // pass, with the events that fork it from and join it to the ctx stream
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int face[6] = {0, 0, 0, 0, 0, 0};  // described boundary faces (StepParams::face)
  bool x_linked = false;             // the x-faces' sources are served by ghost links
  bool x_inlet = false;              // the x = 0 plane is INLET, served by the bulk pass
  bool x_outlet = false;             // the x = nx - 1 plane is OUTLET, served by the bulk pass
  float* link_q = nullptr;  // Bouzidi wall distance per link (LINK_BZ entries), or null
  float* inlet_field = nullptr;  // D * N inlet velocities (xlb_set_inlet_profile), or null
  int inlet_scheme = XLB_INLET_ZOU_HE;
  int inlet_axis = 0, inlet_sign = 1;  // inward normal of the INLET boundary
  bool has_inlet_outlet = false;  // INLET, OUTLET or FWALL cells (no adjoint)
  float* init_fields = nullptr;  // (1 + D) * N: rho0, u0 (component-major)
  bool has_init = false;
  int kind_h = 0;
  int64_t t = 0;
  // boundary values and force
  float lid_rho = 1.f, lid_u[3] = {0, 0, 0};
  float inlet_u[3] = {0, 0, 0};
  float eq_rho = 1.f, eq_u[3] = {0, 0, 0};
  float F[3] = {0, 0, 0};
  bool has_force = false;
  // scratch
  double* partial = nullptr;
  long long partial_cap = 0;
  double* red_out = nullptr;
  int* err_word = nullptr;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // tape / adjoint
  bool tape_open = false;
  int64_t tape_T = 0, tape_k = 0;
  std::vector<void*> ckpt;   // views into the tape arena
  std::vector<void*> slots;
  char* tape_arena = nullptr;  // checkpoints, tape slots and adjoint buffers, kept for reuse
  size_t tape_arena_bytes = 0;
  int64_t seg_loaded = -1;
  float* abar[2] = {nullptr, nullptr};
  int acur = 0;
  int64_t adj_t = -1;  // time index of the adjoint held in abar[acur]
  // kernel variant of the bulk pass (XLB_KERNEL_*)
  int variant = 0;
  // graph replay of the update (xlb_set_step_graph): g updates per graph, one
  // executable graph per starting buffer, each valid for one parameter epoch
  int64_t graph_g = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  uint64_t gexec_epoch[2] = {0, 0};
  uint64_t epoch = 1;  // bumped by every change of the update's parameters
  // profiling
  bool prof = false;
  std::vector<EventPair> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  std::string err;
};

static std::string g_create_err;

static int fail(xlb_ctx* c, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (c)
    c->err = msg;
  else
    g_create_err = msg;
  return code;
}

static int cuda_fail(xlb_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();  // a failed allocation must not surface again at the next launch check
  return fail(c, e == cudaErrorMemoryAllocation ? XLB_ERR_OOM : XLB_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory mapped into the device's address space (what
// cudaHostAlloc / cudaHostRegister give with unified addressing): kernels
// read and write it over the host link themselves, which on this platform
// moves a field faster than a staged copy-engine transfer.  Returns the
// device-side pointer, or null for any other memory.
static void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static size_t state_elems(const xlb_ctx* c) { return (size_t)c->Q * (size_t)c->plane; }
static size_t state_bytes_raw(const xlb_ctx* c) { return state_elems(c) * (size_t)c->esize; }

static int ensure_stage(xlb_ctx* c, size_t bytes) {
  if (c->stage_bytes >= bytes) return XLB_OK;
  if (c->stage) cudaFree(c->stage);
  c->stage = nullptr;
  c->stage_bytes = 0;
  CK(cudaMalloc(&c->stage, bytes));
  c->stage_bytes = bytes;
  return XLB_OK;
}

static StepParams make_params(const xlb_ctx* c) {
  StepParams p;
  memset(&p, 0, sizeof p);
  p.nx = (int)c->nx;
  p.ny = (int)c->ny;
  p.nz = (int)c->nz;
  p.plane = c->plane;
  p.omega = (float)c->omega;
  p.has_mask = c->has_mask ? 1 : 0;
  p.flags = c->flags;
  p.has_force = c->has_force ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    p.F[a] = c->F[a];
    p.eq_u[a] = c->eq_u[a];
    p.inlet_u[a] = c->inlet_u[a];
  }
  if (c->D == 2) {
    p.F[2] = 0.f;
    p.eq_u[2] = 0.f;
    p.inlet_u[2] = 0.f;
  }
  p.eq_rho = c->eq_rho;
  p.inlet_field = c->inlet_field;
  p.inlet_regularized = c->inlet_scheme == XLB_INLET_REGULARIZED;
  p.inlet_axis = c->inlet_axis;
  p.inlet_sign = c->inlet_sign;
  p.err = c->err_word ? c->err_word + 1 : nullptr;
  p.has_faces = 0;
  for (int f = 0; f < 6; ++f) {
    p.face[f] = c->face[f];
    p.has_faces |= c->face[f] != 0;
  }
  p.x_linked = c->x_linked ? 1 : 0;
  p.x_inlet = c->x_inlet ? 1 : 0;
  p.x_outlet = c->x_outlet ? 1 : 0;
  // constant boundary terms per direction, in double then rounded once
  auto fill = [&](auto lat_tag) {
    constexpr int Q = decltype(lat_tag)::value;
    const double eu[3] = {c->eq_u[0], c->eq_u[1], Lattice<Q>::D == 3 ? c->eq_u[2] : 0.0};
    const double lu[3] = {c->lid_u[0], c->lid_u[1], Lattice<Q>::D == 3 ? c->lid_u[2] : 0.0};
    const double usq = eu[0] * eu[0] + eu[1] * eu[1] + eu[2] * eu[2];
    for (int i = 0; i < Q; ++i) {
      const double w = weight_d<Q>(i);
      const double cu = Lattice<Q>::c(i, 0) * eu[0] + Lattice<Q>::c(i, 1) * eu[1] + Lattice<Q>::c(i, 2) * eu[2];
      p.eq_df[i] = (float)(w * (c->eq_rho - 1.0) + w * c->eq_rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
      const double cl = Lattice<Q>::c(i, 0) * lu[0] + Lattice<Q>::c(i, 1) * lu[1] + Lattice<Q>::c(i, 2) * lu[2];
      p.lid_term[i] = (float)(6.0 * w * c->lid_rho * cl);
    }
  };
  if (c->Q == 9) fill(std::integral_constant<int, 9>());
  if (c->Q == 19) fill(std::integral_constant<int, 19>());
  if (c->Q == 27) fill(std::integral_constant<int, 27>());
  return p;
}

static int dispatch(xlb_ctx* c, Op op, const LaunchArgs& a) {
  int r;
  if (c->Q == 9)
    r = launch_d2q9(op, a);
  else if (c->Q == 19)
    r = launch_d3q19(op, a);
  else
    r = launch_d3q27(op, a);
  if (r != 0) return fail(c, XLB_ERR_UNSUPPORTED, "launch of op %d rejected (code %d)", (int)op, r);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return XLB_OK;
}

static LaunchArgs base_args(xlb_ctx* c) {
  LaunchArgs a;
  memset(&a, 0, sizeof a);
  a.p = make_params(c);
  a.storage = c->storage;
  a.coll = c->coll;
  a.ucs = c->N;
  a.stream = c->stream;
  a.partial = c->partial;
  a.partial_capacity = c->partial_cap;
  return a;
}

static cudaEvent_t* prof_begin(xlb_ctx* c, int kind) {
  if (!c->prof) return nullptr;
  if (c->ev_used == c->ev_pool.size()) {
    EventPair e;
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
    c->ev_kind.push_back(kind);
  }
  c->ev_kind[c->ev_used] = kind;
  EventPair& e = c->ev_pool[c->ev_used++];
  cudaEventRecord(e.a, c->stream);
  return &e.b;
}

static void prof_end(xlb_ctx* c, cudaEvent_t* b) {
  if (b) cudaEventRecord(*b, c->stream);
}

// The vectorised bulk kernel (4 cells per thread) runs 16-bit storage with
// BGK or NONE collision on D2Q9 / D3Q19 when nx is a multiple of 4; FP32 is
// fastest with one cell per thread (measured on the 256^3 cavity).
static bool vec_possible(const xlb_ctx* c, int width = 4) {
  return c->esize == 2 && c->Q != 27 && c->coll == XLB_COLL_BGK && c->nx % width == 0;
}

// The vectorised kernel has no full-way reversal for FWALL face planes.
static bool has_fwall_face(const xlb_ctx* c) {
  for (int f = 0; f < 6; ++f)
    if (c->face[f] == XLB_CELL_FWALL) return true;
  return false;
}

// The bulk variant an update launches: the requested one where it can run
// this ctx, and for AUTO the fastest measured on the 256^3 D3Q19 lattices
// (periodic box and cavity): with FP16 storage 4 cells per thread without
// boundary faces (70.4 k MLUPS against 66.3 k for one cell per thread) and 2
// cells per thread with them (59.0 k against 57.3 k); with BF16 storage
// (whose stochastic rounding adds per-value work) and FP32 one cell per
// thread.  Masks with FWALL faces always run one cell per thread.
static int bulk_variant(const xlb_ctx* c) {
  if (c->variant == XLB_KERNEL_DIRECT || has_fwall_face(c)) return XLB_KERNEL_DIRECT;
  if (c->variant == XLB_KERNEL_VEC2) return vec_possible(c, 2) ? XLB_KERNEL_VEC2 : XLB_KERNEL_DIRECT;
  if (c->variant == XLB_KERNEL_VEC) return vec_possible(c, 4) ? XLB_KERNEL_VEC : XLB_KERNEL_DIRECT;
  if (c->storage != XLB_STORE_F16) return XLB_KERNEL_DIRECT;
  bool faces = false;
  for (int f = 0; f < 6; ++f) faces |= c->face[f] != 0;
  if (c->has_mask && c->n_links > 0) faces = true;  // boundary planes served by ghost links
  if (!faces && vec_possible(c, 4)) return XLB_KERNEL_VEC;
  if (vec_possible(c, 2)) return XLB_KERNEL_VEC2;
  return XLB_KERNEL_DIRECT;
}

static bool use_vec(const xlb_ctx* c) { return bulk_variant(c) != XLB_KERNEL_DIRECT; }

// Boundary pass on dst after a pass that produced post-collision values
// there: ghost values of every link and of the inlet / outlet cells' links;
// with `fix_src`, the inlet / outlet cells are first recomputed from it (or,
// with `from_side`, their recomputation is taken from the side buffer).
// Without it (the state came from a local collision or a restore, not from
// the bulk kernel, which pushes them itself), the ghost values of the
// boundary faces are written first.
static int boundary_pass(xlb_ctx* c, const void* fix_src, void* dst, bool from_side = false) {
  if (!c->has_mask) return XLB_OK;
  if (!fix_src) {
    bool faces = false;
    for (int f = 0; f < 6; ++f) faces |= c->face[f] != 0;
    if (faces) {
      LaunchArgs g = base_args(c);
      g.dst = dst;
      const int r = dispatch(c, OP_FACE_GHOSTS, g);
      if (r) return r;
    }
  }
  if (c->n_links + c->n_fix == 0) return XLB_OK;
  LaunchArgs a = base_args(c);
  a.src = fix_src ? fix_src : dst;
  a.dst = dst;
  a.links = c->links;
  a.link_cells = c->link_cells;
  a.link_q = c->link_q;
  a.n_links = c->n_links;
  a.fix = c->fix;
  a.n_fix = c->n_fix;
  a.fix_mode = fix_src ? (from_side ? FIX_SIDE_COMMIT : FIX_RECOMPUTE) : FIX_STORED;
  a.side = c->fix_side;
  return dispatch(c, OP_BOUNDARY, a);
}

// One lattice update from buffer src to dst (either the live pair or tape
// slots): a bulk pass that pulls every cell as if periodic (no flag reads) --
// the wall, lid and EQ cells hold ghost values that make that pull exact;
// whole inlet / outlet x-planes take their rules in the bulk pass too --
// then the boundary pass, which rewrites the ghosts for the next step and
// stores the other fix-up cells (inlet / outlet cells off those planes,
// FWALL cells off the faces).
// The fix-up cells' recomputation reads only src, so it runs on the
// auxiliary stream beside the bulk pass (forked from and joined back to the
// ctx stream by events, which a graph capture turns into parallel branches)
// and leaves its results in the side buffer; the boundary pass after the
// bulk pass stores them and writes their ghost values.  On small lattices
// with many inlet / outlet cells this takes their serial recomputation off
// the critical path.
static int launch_step(xlb_ctx* c, const void* src, void* dst) {
  const bool vec = use_vec(c);
  LaunchArgs a = base_args(c);
  a.src = src;
  a.dst = dst;
  a.vec_width = bulk_variant(c) == XLB_KERNEL_VEC2 ? 2 : 4;
  a.p.has_mask = 0;  // bulk pass: every cell pulled as if periodic
  cudaEvent_t* pe = prof_begin(c, 0);
  const bool side = c->has_mask && c->n_fix > 0 && c->fix_side && c->aux;
  int r = XLB_OK;
  if (side) {
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    LaunchArgs f = base_args(c);
    f.src = src;
    f.dst = dst;
    f.fix = c->fix;
    f.n_fix = c->n_fix;
    f.fix_mode = FIX_SIDE_COMPUTE;
    f.side = c->fix_side;
    f.stream = c->aux;
    r = dispatch(c, OP_BOUNDARY, f);
    cudaError_t e = cudaEventRecord(c->ev_join, c->aux);
    if (!r && e != cudaSuccess) r = cuda_fail(c, e, "cudaEventRecord(join)");
  }
  if (!r) r = dispatch(c, vec ? OP_STEP_VEC : OP_STEP, a);
  if (side) {
    // join even after a failure, so that a capture in progress stays whole
    cudaError_t e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    if (!r && e != cudaSuccess) r = cuda_fail(c, e, "cudaStreamWaitEvent(join)");
  }
  if (!r) r = boundary_pass(c, src, dst, side);
  prof_end(c, pe);
  return r;
}

// Device error word (bounded waits that expired) -> XLB_ERR_TIMEOUT.
static int check_device_error(xlb_ctx* c) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->err_word + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h) {
    CK(cudaMemsetAsync(c->err_word + 1, 0, sizeof(int), c->stream));
    return fail(c, XLB_ERR_TIMEOUT, "a bounded wait inside a kernel expired (device error %d); results are invalid", h);
  }
  return XLB_OK;
}

// Turn a post-collision state h_{t-1} into the post-stream state f_t it
// represents, under the current boundaries (a stream-only update into the
// other buffer).  Used before the boundaries change, so that f_t keeps the
// boundaries it was streamed with and the change acts from step t + 1 on.
static int materialize_post_stream(xlb_ctx* c) {
  if (!c->kind_h) return XLB_OK;
  const int coll = c->coll;
  c->coll = XLB_COLL_NONE;
  const int r = launch_step(c, c->buf[c->cur], c->buf[c->cur ^ 1]);
  c->coll = coll;
  if (r) return r;
  c->cur ^= 1;
  c->kind_h = 0;
  return XLB_OK;
}

static int launch_collide_local(xlb_ctx* c, void* buf) {
  LaunchArgs a = base_args(c);
  a.dst = buf;
  int r = dispatch(c, OP_COLLIDE_LOCAL, a);
  if (!r) r = boundary_pass(c, nullptr, buf);  // ghosts of the first post-collision state
  return r;
}

static int launch_init(xlb_ctx* c, void* dst) {
  LaunchArgs a = base_args(c);
  a.dst = dst;
  a.rho = c->init_fields;
  a.u = c->init_fields + c->N;
  return dispatch(c, OP_INIT, a);
}

// The six boundary planes of a mask, gathered on the device into one compact
// host buffer (the x-planes are strided in the mask): plane f (x = 0,
// x = nx - 1, y = 0, ..., z = nz - 1) holds its cells at a + n1 * b, (a, b)
// the coordinates on the next two axes; axes of extent 1 have none.
struct FacePlanes {
  std::vector<uint8_t> data;
  long long off[6], n1[6];
  int at(int f, long long a, long long b) const { return data[(size_t)(off[f] + a + n1[f] * b)]; }
};

// Boundary faces of a mask (its face planes): a face plane qualifies when none of
// its cells is fluid-like; its type is that of the plane's centre cell.  A
// face stays only while every cell of its plane has the type the pull derives
// from the remaining faces (where planes meet WALL wins, then FWALL; at most
// one other type among LID / EQ); dropped faces are covered by ghost links
// and the fix-up list.  Axes of extent 1 carry no faces.
static void detect_faces(const FacePlanes& pl, long long nx, long long ny, long long nz, int out[6]) {
  for (int f = 0; f < 6; ++f) out[f] = 0;
  const long long ext[3] = {nx, ny, nz};
  auto fl = [](int t) { return t == XLB_CELL_FLUID || t == XLB_CELL_INLET || t == XLB_CELL_OUTLET; };
  int cand[6] = {0, 0, 0, 0, 0, 0};
  for (int f = 0; f < 6; ++f) {
    const int ax = f / 2;
    if (ext[ax] < 2) continue;
    const long long pos = (f % 2) ? ext[ax] - 1 : 0;
    const long long n1 = ext[(ax + 1) % 3], n2 = ext[(ax + 2) % 3];
    (void)pos;
    bool ok = true;
    for (long long b = 0; b < n2 && ok; ++b)
      for (long long a = 0; a < n1 && ok; ++a) ok = !fl(pl.at(f, a, b));
    if (!ok) continue;
    const int t = pl.at(f, n1 / 2, n2 / 2);
    if (t == XLB_CELL_WALL || t == XLB_CELL_LID || t == XLB_CELL_EQ || t == XLB_CELL_FWALL) cand[f] = t;
  }
  int other = 0;
  for (int f = 0; f < 6; ++f)
    if (cand[f] == XLB_CELL_LID || cand[f] == XLB_CELL_EQ) {
      if (other && other != cand[f]) return;
      other = cand[f];
    }
  // verify every cell of every qualifying plane; drop a face whose plane has
  // a cell of another type than the faces derive, and check again
  for (bool changed = true; changed;) {
    changed = false;
    for (int f = 0; f < 6 && !changed; ++f) {
      if (!cand[f]) continue;
      const int ax = f / 2;
      const long long pos = (f % 2) ? ext[ax] - 1 : 0;
      const long long n1 = ext[(ax + 1) % 3], n2 = ext[(ax + 2) % 3];
      bool bad = false;
      for (long long b = 0; b < n2 && !bad; ++b)
        for (long long a = 0; a < n1 && !bad; ++a) {
          // a cell off the plane's border lies on no other face plane
          int want = cand[f];
          if (a == 0 || a == n1 - 1 || b == 0 || b == n2 - 1) {
            long long q[3];
            q[ax] = pos;
            q[(ax + 1) % 3] = a;
            q[(ax + 2) % 3] = b;
            int tw = 0, tf = 0, to = 0;
            for (int g = 0; g < 6; ++g) {
              if (!cand[g]) continue;
              const int gx = g / 2;
              const long long gp = (g % 2) ? ext[gx] - 1 : 0;
              if (q[gx] == gp) {
                if (cand[g] == XLB_CELL_WALL)
                  tw = XLB_CELL_WALL;
                else if (cand[g] == XLB_CELL_FWALL)
                  tf = XLB_CELL_FWALL;
                else
                  to = cand[g];
              }
            }
            want = tw ? tw : (tf ? tf : to);
          }
          bad = pl.at(f, a, b) != want;
        }
      if (bad) {
        cand[f] = 0;
        changed = true;
      }
    }
  }
  for (int f = 0; f < 6; ++f) out[f] = cand[f];
}

template <int Q>
static void fill_lattice(int32_t* c, double* w) {
  for (int i = 0; i < Q; ++i) {
    if (c)
      for (int a = 0; a < 3; ++a) c[3 * i + a] = Lattice<Q>::c(i, a);
    if (w) w[i] = weight_d<Q>(i);
  }
}

extern "C" {

const char* xlb_status_string(int s) {
  switch (s) {
    case XLB_OK: return "XLB_OK";
    case XLB_ERR_ARG: return "XLB_ERR_ARG";
    case XLB_ERR_UNSUPPORTED: return "XLB_ERR_UNSUPPORTED";
    case XLB_ERR_OOM: return "XLB_ERR_OOM";
    case XLB_ERR_CUDA: return "XLB_ERR_CUDA";
    case XLB_ERR_TIMEOUT: return "XLB_ERR_TIMEOUT";
    case XLB_ERR_STATE: return "XLB_ERR_STATE";
    default: return "XLB_ERR_UNKNOWN";
  }
}

const char* xlb_last_error(const xlb_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

double xlb_omega_from_nu(double nu) { return 1.0 / (3.0 * nu + 0.5); }

int xlb_create(xlb_ctx** out, int lattice, const int64_t dims[3], double omega, int collision, int storage,
               void* cuda_stream) {
  if (!out) return fail(nullptr, XLB_ERR_ARG, "out is null");
  *out = nullptr;
  if (lattice != 9 && lattice != 19 && lattice != 27) return fail(nullptr, XLB_ERR_ARG, "lattice must be 9, 19 or 27");
  if (!dims) return fail(nullptr, XLB_ERR_ARG, "dims is null");
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, XLB_ERR_ARG, "dims must be >= 1");
  if (lattice == 9 && nz != 1) return fail(nullptr, XLB_ERR_ARG, "D2Q9 needs nz = 1");
  if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30) || nx * ny > (1LL << 40) || nx * ny * nz > (1LL << 40))
    return fail(nullptr, XLB_ERR_ARG, "dims too large");
  if (nx * ny * nz > 0x7fffffffLL)
    return fail(nullptr, XLB_ERR_UNSUPPORTED, "at most 2^31 - 1 cells per lattice (32-bit cell indices)");
  if (!(omega > 0.0 && omega < 2.0)) return fail(nullptr, XLB_ERR_ARG, "omega must lie in (0, 2)");
  if (collision < 0 || collision > 2) return fail(nullptr, XLB_ERR_ARG, "unknown collision %d", collision);
  if (collision == XLB_COLL_KBC && lattice == 19)
    return fail(nullptr, XLB_ERR_UNSUPPORTED, "KBC is defined on D2Q9 and D3Q27 only");
  if (storage < 0 || storage > 2) return fail(nullptr, XLB_ERR_ARG, "unknown storage %d", storage);

  xlb_ctx* c = new xlb_ctx();
  c->Q = lattice;
  c->D = lattice == 9 ? 2 : 3;
  c->coll = collision;
  c->storage = storage;
  c->esize = storage == XLB_STORE_F32 ? 4 : 2;
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->N = nx * ny * nz;
  // population planes start on 256-byte boundaries
  const long long align = 256 / c->esize;
  c->plane = (c->N + align - 1) / align * align;
  c->omega = omega;
  auto bail = [&](int code) {
    g_create_err = c->err;
    xlb_destroy(c);
    return code;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
    c->own_stream = true;
  }
  for (int k = 0; k < 2; ++k) {
    e = cudaMalloc(&c->buf[k], state_bytes_raw(c));
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(populations)"));
  }
  StepParams p = make_params(c);
  c->partial_cap = row_blocks(p);
  e = cudaMalloc(&c->partial, sizeof(double) * 4 * (size_t)(c->partial_cap > 0 ? c->partial_cap : 1));
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(partials)"));
  e = cudaMalloc(&c->red_out, 4 * sizeof(double) + sizeof(int) * 4);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(reduction)"));
  c->err_word = (int*)(c->red_out + 4);
  e = cudaMemset(c->err_word, 0, 4 * sizeof(int));
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemset(error words)"));
  e = cudaMalloc(&c->init_fields, sizeof(float) * (size_t)(1 + c->D) * (size_t)c->N);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(init fields)"));
  e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "auxiliary stream"));
  *out = c;
  return XLB_OK;
}

int xlb_tape_end(xlb_ctx* c);

int xlb_tape_release(xlb_ctx* c);

void xlb_destroy(xlb_ctx* c) {
  if (!c) return;
  xlb_tape_release(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int k = 0; k < 2; ++k)
    if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
  for (int k = 0; k < 2; ++k)
    if (c->buf[k]) cudaFree(c->buf[k]);
  if (c->flags) cudaFree(c->flags);
  if (c->links) cudaFree(c->links);
  if (c->link_cells) cudaFree(c->link_cells);
  if (c->link_q) cudaFree(c->link_q);
  if (c->inlet_field) cudaFree(c->inlet_field);
  if (c->fix) cudaFree(c->fix);
  if (c->init_fields) cudaFree(c->init_fields);
  if (c->fix_side) cudaFree(c->fix_side);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->partial) cudaFree(c->partial);
  if (c->red_out) cudaFree(c->red_out);
  if (c->stage) cudaFree(c->stage);
  for (auto& e : c->ev_pool) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// Inflow / outflow x-planes served by the bulk pass: the x = 0 plane whose
// cells are all INLET, and the x = nx - 1 plane whose cells are all OUTLET,
// apart from the cells on the y / z face planes (which the faces describe).
// The bulk pass then applies the inlet rule in the lanes of x = 0 and, in the
// lanes of x = nx - 1, pulls the directions c_x = -1 as x - 1 does (their
// sources lie in the cell's own column), and those cells leave the fix-up
// list: the strided x-planes are then written only by the coalesced rows of
// the bulk pass.
static void detect_io_planes(const FacePlanes& pl, long long nx, long long ny, long long nz, const int face[6],
                             bool* x_in, bool* x_out) {
  *x_in = *x_out = false;
  if (nx < 3) return;
  bool in_ok = true, out_ok = true, any = false;
  for (long long z = 0; z < nz && (in_ok || out_ok); ++z)
    for (long long y = 0; y < ny && (in_ok || out_ok); ++y) {
      const bool on_yz = (y == 0 && face[2]) || (y == ny - 1 && face[3]) || (nz > 1 && z == 0 && face[4]) ||
                         (nz > 1 && z == nz - 1 && face[5]);
      if (on_yz) continue;
      any = true;
      in_ok = in_ok && pl.at(0, y, z) == XLB_CELL_INLET;
      out_ok = out_ok && pl.at(1, y, z) == XLB_CELL_OUTLET;
    }
  *x_in = any && in_ok;
  *x_out = any && out_ok;
}

int xlb_set_mask(xlb_ctx* c, const uint8_t* mask) {
  if (!c) return XLB_ERR_ARG;
  if (!mask) return fail(c, XLB_ERR_ARG, "mask is null");
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "the mask cannot change while a tape is open");
  const size_t n = (size_t)c->N;
  uint8_t* dmask = nullptr;
  bool host_mask = !is_device_ptr(mask);
  if (host_mask) {
    int r = ensure_stage(c, n);
    if (r) return r;
    CK(cudaMemcpyAsync(c->stage, mask, n, cudaMemcpyHostToDevice, c->stream));
    dmask = (uint8_t*)c->stage;
  } else {
    dmask = (uint8_t*)mask;
  }
  uint8_t* nf = nullptr;
  bool new_io = false, new_x_inlet = false, new_x_outlet = false;
  int new_face[6] = {0, 0, 0, 0, 0, 0};
  CK(cudaMalloc(&nf, n));
  CK(cudaMemsetAsync(c->err_word, 0, sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->err_word + 2, 0, sizeof(int), c->stream));
  if (launch_mask_prepare(c->Q, dmask, nf, (int)c->nx, (int)c->ny, (int)c->nz, c->err_word, c->stream) != 0) {
    cudaFree(nf);
    return fail(c, XLB_ERR_ARG, "mask preparation rejected");
  }
  int hw[3] = {0, 0, 0};  // bad code; the device error word (not used here); inlet / outlet / FWALL seen
  CK(cudaMemcpyAsync(hw, c->err_word, sizeof(hw), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int herr = hw[0];
  if (herr) {
    cudaFree(nf);
    return fail(c, XLB_ERR_ARG, "mask holds a code >= 7");
  }
  // inlet / outlet / FWALL cells anywhere (the adjoint support check), from
  // the preparation kernel; the boundary faces, from the mask's face planes
  {
    FacePlanes pl;
    const long long ext[3] = {c->nx, c->ny, c->nz};
    long long tot = 0;
    for (int f = 0; f < 6; ++f) {
      const int ax = f / 2;
      pl.off[f] = tot;
      pl.n1[f] = ext[(ax + 1) % 3];
      if (ext[ax] >= 2) tot += ext[(ax + 1) % 3] * ext[(ax + 2) % 3];
    }
    pl.data.resize((size_t)tot);
    if (tot > 0) {
      uint8_t* dp = nullptr;
      CK(cudaMalloc(&dp, (size_t)tot));
      cudaError_t e = launch_extract_planes(dmask, (int)c->nx, (int)c->ny, (int)c->nz, dp, c->stream) != 0
                          ? cudaErrorInvalidValue
                          : cudaMemcpyAsync(pl.data.data(), dp, (size_t)tot, cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      cudaFree(dp);
      if (e != cudaSuccess) {
        cudaFree(nf);
        return cuda_fail(c, e, "face planes");
      }
    }
    new_io = hw[2] != 0;
    detect_faces(pl, c->nx, c->ny, c->nz, new_face);
    bool fw_face = false;  // (the bulk instance for FWALL faces has no inflow / outflow planes)
    for (int f = 0; f < 6; ++f) fw_face |= new_face[f] == XLB_CELL_FWALL;
    if (new_io && !fw_face) detect_io_planes(pl, c->nx, c->ny, c->nz, new_face, &new_x_inlet, &new_x_outlet);
  }
  // With 16-bit storage the bulk pass is bound by instruction issue, and the
  // x-face rules would run in diverging lanes at both ends of every row: the
  // sources on WALL / LID / EQ x-face planes (outside the skipped y / z face
  // rows) go to the ghost links instead, written by the boundary pass after
  // each update.  The x-faces still take part in deriving the rule of the
  // cells where planes meet.  Lattices with an FWALL x-face keep the rules in
  // the pull.  (Two forms that write these values from the bulk pass itself
  // measured slower on the FP16 256^3 cavity: ghost values held in each
  // row's face cell, 55.7 k against 59.9 k MLUPS, and ghost values pushed by
  // the cells next to the faces, 57.9 k against 58.7 k: both diverge the
  // lanes at the row ends.)
  const bool new_x_linked = c->esize == 2 && (new_face[0] || new_face[1]) && new_face[0] != XLB_CELL_FWALL &&
                            new_face[1] != XLB_CELL_FWALL;
  int link_face[6];
  for (int f = 0; f < 6; ++f) link_face[f] = (new_x_linked && f < 2) ? 0 : new_face[f];
  // boundary tables: ghost links (direction-major) and inlet / outlet cells
  int2* nlinks = nullptr;
  int2* nlcells = nullptr;
  int* nfix = nullptr;
  long long nl = 0, nfx = 0;
  {
    const long long nb = bnd_list_blocks(c->N);
    int* counts = nullptr;
    long long* offs = nullptr;
    cudaError_t e = cudaMalloc(&counts, sizeof(int) * nb * (c->Q + 1));
    if (e == cudaSuccess) e = cudaMalloc(&offs, sizeof(long long) * nb * (c->Q + 1));
    std::vector<int> hc(nb * (c->Q + 1));
    std::vector<long long> ho(nb * (c->Q + 1));
    // passes 1..Q-1: links of direction i; pass Q: inlet / outlet cells
    if (e == cudaSuccess && launch_pred_count(c->Q, link_face, new_x_inlet, new_x_outlet, nf, (int)c->nx,
                                              (int)c->ny, (int)c->nz, counts, c->stream) != 0)
      e = cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hc.data() + nb, counts + nb, sizeof(int) * nb * c->Q, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
      for (int pass = 1; pass <= c->Q; ++pass) {
        long long& run = pass == c->Q ? nfx : nl;
        for (long long b = 0; b < nb; ++b) {
          ho[nb * pass + b] = run;
          run += hc[nb * pass + b];
        }
      }
      e = cudaMemcpyAsync(offs + nb, ho.data() + nb, sizeof(long long) * nb * c->Q, cudaMemcpyHostToDevice,
                          c->stream);
    }
    if (e == cudaSuccess && nl > 0) e = cudaMalloc(&nlinks, sizeof(int2) * nl);
    if (e == cudaSuccess && nl > 0) e = cudaMalloc(&nlcells, sizeof(int2) * nl);
    if (e == cudaSuccess && nfx > 0) e = cudaMalloc(&nfix, sizeof(int) * nfx);
    if (e == cudaSuccess && nl + nfx > 0 &&
        launch_pred_write(c->Q, link_face, new_x_inlet, new_x_outlet, nf, (int)c->nx, (int)c->ny, (int)c->nz, offs,
                          nlinks, nfix, c->stream) != 0)
      e = cudaErrorInvalidValue;
    if (e == cudaSuccess && nl > 0 &&
        launch_link_cells(c->Q, nlinks, nl, nf, (int)c->nx, (int)c->ny, (int)c->nz, nlcells, c->stream) != 0)
      e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (counts) cudaFree(counts);
    if (offs) cudaFree(offs);
    if (e != cudaSuccess) {
      cudaFree(nf);
      if (nlinks) cudaFree(nlinks);
      if (nlcells) cudaFree(nlcells);
      if (nfix) cudaFree(nfix);
      return cuda_fail(c, e, "boundary tables");
    }
  }
  {
    const int r = materialize_post_stream(c);  // f_t under the old mask
    if (r) {
      cudaFree(nf);
      if (nlinks) cudaFree(nlinks);
      if (nlcells) cudaFree(nlcells);
      if (nfix) cudaFree(nfix);
      return r;
    }
  }
  void* nside = nullptr;
  if (nfx > 0) {
    const cudaError_t e = cudaMalloc(&nside, (size_t)c->esize * (size_t)c->Q * (size_t)nfx);
    if (e != cudaSuccess) {
      cudaFree(nf);
      if (nlinks) cudaFree(nlinks);
      if (nlcells) cudaFree(nlcells);
      if (nfix) cudaFree(nfix);
      return cuda_fail(c, e, "cudaMalloc(fix-up side buffer)");
    }
  }
  if (c->flags) cudaFree(c->flags);
  if (c->links) cudaFree(c->links);
  if (c->link_cells) cudaFree(c->link_cells);
  if (c->link_q) cudaFree(c->link_q);
  c->link_q = nullptr;  // wall distances belong to the old link table
  if (c->fix_side) cudaFree(c->fix_side);
  c->fix_side = nside;
  if (c->fix) cudaFree(c->fix);
  c->flags = nf;
  c->links = nlinks;
  c->link_cells = nlcells;
  c->n_links = nl;
  c->fix = nfix;
  c->n_fix = nfx;
  c->has_inlet_outlet = new_io;
  for (int f = 0; f < 6; ++f) c->face[f] = new_face[f];
  c->x_linked = new_x_linked;
  c->x_inlet = new_x_inlet;
  c->x_outlet = new_x_outlet;
  c->has_mask = true;
  ++c->epoch;
  return XLB_OK;
}

int xlb_lattice_table(int lattice, int32_t* c, double* w) {
  if (lattice == 9)
    fill_lattice<9>(c, w);
  else if (lattice == 19)
    fill_lattice<19>(c, w);
  else if (lattice == 27)
    fill_lattice<27>(c, w);
  else
    return XLB_ERR_ARG;
  return XLB_OK;
}

static int lattice_opposite(int Q, int i) {
  return Q == 9 ? opposite<9>(i) : (Q == 19 ? opposite<19>(i) : opposite<27>(i));
}

int xlb_set_inlet_profile(xlb_ctx* c, const float* u) {
  if (!c) return XLB_ERR_ARG;
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "boundary values cannot change while a tape is open");
  const int r = materialize_post_stream(c);  // f_t with the old inlet
  if (r) return r;
  if (!u) {
    if (c->inlet_field) CK(cudaFree(c->inlet_field));
    c->inlet_field = nullptr;
    ++c->epoch;
    return XLB_OK;
  }
  const size_t bytes = sizeof(float) * (size_t)c->D * (size_t)c->N;
  if (!c->inlet_field) CK(cudaMalloc(&c->inlet_field, bytes));
  CK(cudaMemcpyAsync(c->inlet_field, u, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  ++c->epoch;
  return XLB_OK;
}

int xlb_set_inlet_scheme(xlb_ctx* c, int scheme) {
  if (!c) return XLB_ERR_ARG;
  if (scheme != XLB_INLET_ZOU_HE && scheme != XLB_INLET_REGULARIZED)
    return fail(c, XLB_ERR_ARG, "unknown inlet scheme %d", scheme);
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "boundary values cannot change while a tape is open");
  const int r = materialize_post_stream(c);  // f_t with the old rule
  if (r) return r;
  c->inlet_scheme = scheme;
  ++c->epoch;
  return XLB_OK;
}

int xlb_set_inlet_normal(xlb_ctx* c, int axis, int sign) {
  if (!c) return XLB_ERR_ARG;
  if (axis < 0 || axis >= c->D || (sign != 1 && sign != -1))
    return fail(c, XLB_ERR_ARG, "normal: axis in [0, %d), sign +1 or -1", c->D);
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "boundary values cannot change while a tape is open");
  const int r = materialize_post_stream(c);  // f_t with the old normal
  if (r) return r;
  c->inlet_axis = axis;
  c->inlet_sign = sign;
  ++c->epoch;
  return XLB_OK;
}

int xlb_set_wall_distances(xlb_ctx* c, int64_t n, const int64_t* cell, const int32_t* dir, const float* q) {
  if (!c) return XLB_ERR_ARG;
  if (n < 0 || (n > 0 && (!cell || !dir || !q))) return fail(c, XLB_ERR_ARG, "n < 0 or a null array");
  if (!c->has_mask) return fail(c, XLB_ERR_STATE, "set a mask first");
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "boundary values cannot change while a tape is open");
  // host copy of the link table; entries of one pulled direction are
  // contiguous and ascending in the cell index
  std::vector<int2> hl((size_t)c->n_links);
  if (c->n_links > 0)
    CK(cudaMemcpy(hl.data(), c->links, sizeof(int2) * hl.size(), cudaMemcpyDeviceToHost));
  for (auto& e : hl) e.y &= ~LINK_BZ;
  std::vector<long long> beg(c->Q + 1, 0);
  {
    long long k = 0;
    for (int j = 0; j <= c->Q; ++j) {
      while (k < (long long)hl.size() && (hl[k].y & 0xff) < j) ++k;
      beg[j] = k;
    }
  }
  std::vector<float> hq(hl.size(), 0.f);
  for (int64_t k = 0; k < n; ++k) {
    const int i = dir[k];
    if (i < 1 || i >= c->Q) return fail(c, XLB_ERR_ARG, "link %lld: direction %d out of range", (long long)k, i);
    if (!(q[k] >= 0.f && q[k] <= 1.f)) return fail(c, XLB_ERR_ARG, "link %lld: q must be in [0, 1]", (long long)k);
    if (cell[k] < 0 || cell[k] >= c->N) return fail(c, XLB_ERR_ARG, "link %lld: cell out of range", (long long)k);
    // the link is pulled in the opposite direction j from the wall cell
    const int j = lattice_opposite(c->Q, i);
    const int2* lo = hl.data() + beg[j];
    const int2* hi = hl.data() + beg[j + 1];
    const int2* e = std::lower_bound(lo, hi, (int)cell[k], [](const int2& a, int v) { return a.x < v; });
    if (e == hi || e->x != (int)cell[k] || ((e->y >> 8) & 0xff) != XLB_CELL_WALL)
      return fail(c, XLB_ERR_ARG,
                  "link %lld (cell %lld, direction %d) is not a ghost link from a FLUID cell to a WALL cell "
                  "off the boundary faces",
                  (long long)k, (long long)cell[k], i);
    const size_t idx = (size_t)(e - hl.data());
    hl[idx].y |= LINK_BZ;
    hq[idx] = q[k];
  }
  // the new rule acts from the next step on (like xlb_set_bc)
  int r = materialize_post_stream(c);
  if (r) return r;
  if (c->link_q) CK(cudaFree(c->link_q));
  c->link_q = nullptr;
  if (n > 0) CK(cudaMalloc(&c->link_q, sizeof(float) * hq.size()));
  if (n > 0) CK(cudaMemcpy(c->link_q, hq.data(), sizeof(float) * hq.size(), cudaMemcpyHostToDevice));
  if (!hl.empty()) CK(cudaMemcpy(c->links, hl.data(), sizeof(int2) * hl.size(), cudaMemcpyHostToDevice));
  ++c->epoch;
  return XLB_OK;
}

int xlb_wall_force(xlb_ctx* c, double* out) {
  if (!c || !out) return XLB_ERR_ARG;
  if (!c->kind_h) return fail(c, XLB_ERR_STATE, "no post-collision state yet: take a step first");
  LaunchArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.links = c->links;
  a.n_links = c->has_mask ? c->n_links : 0;
  long long b = (a.n_links + 255) / 256;
  if (b > c->partial_cap) b = c->partial_cap;
  if (b < 1) b = 1;
  a.partial_capacity = b;
  int r = dispatch(c, OP_WALL_FORCE, a);
  if (r) return r;
  launch_reduce_final(c->partial, b, c->red_out, c->stream);
  if (is_device_ptr(out)) {
    CK(cudaMemcpyAsync(out, c->red_out, 3 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return XLB_OK;
  }
  double h[4];
  CK(cudaMemcpyAsync(h, c->red_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 3; ++k) out[k] = h[k];
  return XLB_OK;
}

int xlb_boundary_links(const xlb_ctx* c, int64_t* n_links, int64_t* n_fix) {
  if (!c || !n_links || !n_fix) return XLB_ERR_ARG;
  *n_links = c->n_links;
  *n_fix = c->n_fix;
  return XLB_OK;
}

int xlb_set_bc(xlb_ctx* c, int type, float rho, const float u[3]) {
  if (!c) return XLB_ERR_ARG;
  if (!u) return fail(c, XLB_ERR_ARG, "u is null");
  if (type != XLB_CELL_LID && type != XLB_CELL_INLET && type != XLB_CELL_EQ)
    return fail(c, XLB_ERR_ARG, "cell type %d carries no boundary value", type);
  if (type == XLB_CELL_INLET && !(u[0] < 1.0f)) return fail(c, XLB_ERR_ARG, "inlet u_x must be < 1");
  if (type == XLB_CELL_EQ && !(rho > 0.f)) return fail(c, XLB_ERR_ARG, "EQ density must be > 0");
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "boundary values cannot change while a tape is open");
  const int r = materialize_post_stream(c);  // f_t with the old values
  if (r) return r;
  if (type == XLB_CELL_LID) {
    c->lid_rho = rho;
    for (int a = 0; a < 3; ++a) c->lid_u[a] = u[a];
  } else if (type == XLB_CELL_INLET) {
    for (int a = 0; a < 3; ++a) c->inlet_u[a] = u[a];
  } else {
    c->eq_rho = rho;
    for (int a = 0; a < 3; ++a) c->eq_u[a] = u[a];
  }
  ++c->epoch;
  return XLB_OK;
}

int xlb_set_force(xlb_ctx* c, const float F[3]) {
  if (!c) return XLB_ERR_ARG;
  if (!F) return fail(c, XLB_ERR_ARG, "F is null");
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "the force cannot change while a tape is open");
  for (int a = 0; a < 3; ++a) c->F[a] = (a < c->D) ? F[a] : 0.f;
  c->has_force = (c->F[0] != 0.f || c->F[1] != 0.f || c->F[2] != 0.f);
  ++c->epoch;
  return XLB_OK;
}

int xlb_init(xlb_ctx* c, const float* rho, const float* u) {
  if (!c) return XLB_ERR_ARG;
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "a tape is open; call xlb_tape_end first");
  const size_t n = (size_t)c->N;
  float* dr = c->init_fields;
  float* du = c->init_fields + n;
  // copy the caller's fields into the library-owned init fields (mapped
  // page-locked host memory: by a copy kernel that reads it directly)
  void* mr = mapped_host_ptr(rho);
  void* mu = mapped_host_ptr(u);
  if (rho && mr) {
    if (launch_copy_f32((const float*)mr, dr, (long long)n, c->stream) != 0) return fail(c, XLB_ERR_CUDA, "copy");
  } else if (rho) {
    CK(cudaMemcpyAsync(dr, rho, n * sizeof(float), cudaMemcpyDefault, c->stream));
  } else {
    std::vector<float> ones(n, 1.0f);
    CK(cudaMemcpyAsync(dr, ones.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (u && mu) {
    if (launch_copy_f32((const float*)mu, du, (long long)c->D * (long long)n, c->stream) != 0)
      return fail(c, XLB_ERR_CUDA, "copy");
  } else if (u) {
    CK(cudaMemcpyAsync(du, u, (size_t)c->D * n * sizeof(float), cudaMemcpyDefault, c->stream));
  } else {
    CK(cudaMemsetAsync(du, 0, (size_t)c->D * n * sizeof(float), c->stream));
  }
  if (!is_device_ptr(rho ? (const void*)rho : (const void*)u)) CK(cudaStreamSynchronize(c->stream));
  c->has_init = true;
  int r = launch_init(c, c->buf[c->cur]);
  if (r) return r;
  c->kind_h = 0;
  c->t = 0;
  return XLB_OK;
}

static int record_checkpoint(xlb_ctx* c) {
  if (!c->tape_open || c->tape_k <= 0) return XLB_OK;
  if (c->t % c->tape_k == 0 && c->t < c->tape_T) {
    const size_t s = (size_t)(c->t / c->tape_k) - 1;
    if (s < c->ckpt.size())
      CK(cudaMemcpyAsync(c->ckpt[s], c->buf[c->cur], state_bytes_raw(c), cudaMemcpyDeviceToDevice, c->stream));
  }
  return XLB_OK;
}

// Executable graph of graph_g updates starting from buffer `from`, captured
// on the ctx stream with the current parameters (recaptured when the epoch
// has moved on).  The graph holds exactly the launches launch_step makes.
static int step_graph(xlb_ctx* c, int from, cudaGraphExec_t* out) {
  if (c->gexec[from] && c->gexec_epoch[from] == c->epoch) {
    *out = c->gexec[from];
    return XLB_OK;
  }
  if (c->gexec[from]) {
    cudaGraphExecDestroy(c->gexec[from]);
    c->gexec[from] = nullptr;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(c->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(c, XLB_ERR_STATE, "the ctx stream is already capturing");
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int cur = from, r = XLB_OK;
  for (int64_t k = 0; k < c->graph_g && r == XLB_OK; ++k) {
    r = launch_step(c, c->buf[cur], c->buf[cur ^ 1]);
    cur ^= 1;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (r != XLB_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return r != XLB_OK ? r : cuda_fail(c, e, "stream capture of the update");
  }
  const cudaError_t ei = cudaGraphInstantiate(&c->gexec[from], g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    c->gexec[from] = nullptr;
    return cuda_fail(c, ei, "cudaGraphInstantiate");
  }
  c->gexec_epoch[from] = c->epoch;
  *out = c->gexec[from];
  return XLB_OK;
}

int xlb_set_step_graph(xlb_ctx* c, int64_t steps_per_graph) {
  if (!c) return XLB_ERR_ARG;
  if (steps_per_graph < 0 || steps_per_graph > 100000)
    return fail(c, XLB_ERR_ARG, "steps_per_graph must be in [0, 100000]");
  if (steps_per_graph != c->graph_g) {
    for (int k = 0; k < 2; ++k)
      if (c->gexec[k]) {
        CK(cudaGraphExecDestroy(c->gexec[k]));
        c->gexec[k] = nullptr;
      }
  }
  c->graph_g = steps_per_graph;
  return XLB_OK;
}

int xlb_step(xlb_ctx* c, int64_t n) {
  if (!c) return XLB_ERR_ARG;
  if (n < 0) return fail(c, XLB_ERR_ARG, "n must be >= 0");
  if (!c->has_init && c->t == 0 && !c->kind_h) return fail(c, XLB_ERR_STATE, "xlb_init (or xlb_state_set) first");
  if (c->tape_open && c->t + n > c->tape_T)
    return fail(c, XLB_ERR_STATE, "stepping past the tape length %lld", (long long)c->tape_T);
  for (int64_t k = 0; k < n; ++k) {
    int r;
    if (c->kind_h && c->graph_g > 0 && !c->tape_open && !c->prof && n - k >= c->graph_g) {
      cudaGraphExec_t ge = nullptr;
      r = step_graph(c, c->cur, &ge);
      if (r) return r;
      CK(cudaGraphLaunch(ge, c->stream));
      if (c->graph_g & 1) c->cur ^= 1;
      c->t += c->graph_g;
      k += c->graph_g - 1;
      continue;
    }
    if (!c->kind_h) {
      r = launch_collide_local(c, c->buf[c->cur]);
      c->kind_h = 1;
    } else {
      r = launch_step(c, c->buf[c->cur], c->buf[c->cur ^ 1]);
      c->cur ^= 1;
    }
    if (r) return r;
    c->t += 1;
    r = record_checkpoint(c);
    if (r) return r;
  }
  return XLB_OK;
}

int xlb_get_time(const xlb_ctx* c, int64_t* t) {
  if (!c || !t) return XLB_ERR_ARG;
  *t = c->t;
  return XLB_OK;
}

int xlb_synchronize(xlb_ctx* c) {
  if (!c) return XLB_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

int xlb_set_kernel(xlb_ctx* c, int variant) {
  if (!c) return XLB_ERR_ARG;
  if (variant < XLB_KERNEL_AUTO || variant > XLB_KERNEL_VEC2)
    return fail(c, XLB_ERR_ARG, "unknown kernel variant %d", variant);
  if (variant == XLB_KERNEL_VEC && !vec_possible(c))
    return fail(c, XLB_ERR_UNSUPPORTED,
                "the vectorised kernel needs 16-bit storage, D2Q9 or D3Q19, BGK and nx %% 4 == 0");
  if (variant == XLB_KERNEL_VEC2 && !vec_possible(c, 2))
    return fail(c, XLB_ERR_UNSUPPORTED,
                "the 2-wide vectorised kernel needs 16-bit storage, D2Q9 or D3Q19, BGK and even nx");
  c->variant = variant;
  ++c->epoch;
  return XLB_OK;
}

int xlb_get_kernel(const xlb_ctx* c, int* variant) {
  if (!c || !variant) return XLB_ERR_ARG;
  *variant = bulk_variant(c);
  return XLB_OK;
}

int xlb_macroscopic(xlb_ctx* c, float* rho, float* u) {
  if (!c) return XLB_ERR_ARG;
  if (!rho && !u) return XLB_OK;
  const size_t n = (size_t)c->N;
  bool host = !is_device_ptr(rho ? (void*)rho : (void*)u);
  float* dr = rho;
  float* du = u;
  // mapped page-locked host memory: the readout kernel writes it directly
  float* mr = (float*)mapped_host_ptr(rho);
  float* mu = (float*)mapped_host_ptr(u);
  if (host && (!rho || mr) && (!u || mu)) {
    dr = mr;
    du = mu;
    host = false;  // nothing to copy; check_device_error below synchronises the stream
  }
  if (host) {
    int r = ensure_stage(c, (1 + c->D) * n * sizeof(float));
    if (r) return r;
    dr = rho ? (float*)c->stage : nullptr;
    du = u ? (float*)c->stage + n : nullptr;
  }
  LaunchArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.kind_h = c->kind_h;
  a.rho_out = dr;
  a.u_out = du;
  int r = dispatch(c, OP_MACRO, a);
  if (r) return r;
  r = check_device_error(c);
  if (r) return r;
  if (host) {
    if (rho) CK(cudaMemcpyAsync(rho, dr, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (u) CK(cudaMemcpyAsync(u, du, (size_t)c->D * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return XLB_OK;
}

int xlb_reduce(xlb_ctx* c, double out_mass[1], double out_mom[3]) {
  if (!c) return XLB_ERR_ARG;
  if (!out_mass && !out_mom) return XLB_OK;
  LaunchArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.kind_h = c->kind_h;
  long long b = (c->N + 127) / 128;
  if (b > c->partial_cap) b = c->partial_cap;
  if (b < 1) b = 1;
  a.partial_capacity = b;
  int r = dispatch(c, OP_REDUCE_PARTIAL, a);
  if (r) return r;
  launch_reduce_final(c->partial, b, c->red_out, c->stream);
  double h[4];
  CK(cudaMemcpyAsync(h, c->red_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  r = check_device_error(c);
  if (r) return r;
  if (out_mass) out_mass[0] = h[0];
  if (out_mom)
    for (int k = 0; k < 3; ++k) out_mom[k] = h[1 + k];
  return XLB_OK;
}

// Box [lo, hi) of a kinetic-energy loss: per axis 0 <= lo < hi <= extent
// (z: 0 and 1 on D2Q9).
static int check_box(xlb_ctx* c, const int64_t lo[3], const int64_t hi[3]) {
  if (!lo || !hi) return fail(c, XLB_ERR_ARG, "box bounds are null");
  const int64_t ext[3] = {c->nx, c->ny, c->nz};
  for (int a = 0; a < 3; ++a)
    if (lo[a] < 0 || hi[a] <= lo[a] || hi[a] > ext[a])
      return fail(c, XLB_ERR_ARG, "box axis %d: need 0 <= lo < hi <= %lld", a, (long long)ext[a]);
  return XLB_OK;
}

// Copy the FP64 result in red_out[0] to out: a device pointer asynchronously
// on the ctx stream, a host pointer synchronously.
static int deliver_scalar(xlb_ctx* c, double* out) {
  if (is_device_ptr(out)) {
    CK(cudaMemcpyAsync(out, c->red_out, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return XLB_OK;
  }
  double h[4];
  CK(cudaMemcpyAsync(h, c->red_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  int r = check_device_error(c);
  if (r) return r;
  out[0] = h[0];
  return XLB_OK;
}

int xlb_kinetic_energy(xlb_ctx* c, const int64_t box_lo[3], const int64_t box_hi[3], double* out) {
  if (!c) return XLB_ERR_ARG;
  if (!out) return fail(c, XLB_ERR_ARG, "out is null");
  int r = check_box(c, box_lo, box_hi);
  if (r) return r;
  LaunchArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.kind_h = c->kind_h;
  for (int k = 0; k < 3; ++k) {
    a.box_lo[k] = (int)box_lo[k];
    a.box_ext[k] = (int)(box_hi[k] - box_lo[k]);
  }
  const long long nbox = (long long)a.box_ext[0] * a.box_ext[1] * a.box_ext[2];
  long long b = (nbox + 127) / 128;
  if (b > c->partial_cap) b = c->partial_cap;
  if (b < 1) b = 1;
  a.partial_capacity = b;
  r = dispatch(c, OP_KE_PARTIAL, a);
  if (r) return r;
  launch_reduce_final(c->partial, b, c->red_out, c->stream);
  return deliver_scalar(c, out);
}

int xlb_sum_squares(xlb_ctx* c, const float* x, int64_t n, double* out) {
  if (!c) return XLB_ERR_ARG;
  if (!x || !out || n < 0) return fail(c, XLB_ERR_ARG, "x or out is null, or n < 0");
  if (n > 0 && !is_device_ptr(x)) return fail(c, XLB_ERR_ARG, "x must be device memory");
  const long long b = launch_sum_squares(x, n, c->partial, c->partial_cap > 0 ? c->partial_cap : 1, c->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "sum of squares launch");
  launch_reduce_final(c->partial, b, c->red_out, c->stream);
  return deliver_scalar(c, out);
}

// Serialized state: 64-byte header then the raw population buffer.
struct StateHeader {
  char magic[8];
  int32_t Q, storage;
  int64_t nx, ny, nz, t;
  int32_t kind_h, reserved;
};
static_assert(sizeof(StateHeader) <= 64, "header");

int xlb_state_bytes(const xlb_ctx* c, size_t* bytes) {
  if (!c || !bytes) return XLB_ERR_ARG;
  *bytes = 64 + state_bytes_raw(c);
  return XLB_OK;
}

int xlb_state_get(xlb_ctx* c, void* buf, size_t bytes) {
  if (!c || !buf) return XLB_ERR_ARG;
  if (bytes < 64 + state_bytes_raw(c)) return fail(c, XLB_ERR_ARG, "buffer too small");
  StateHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, "XLBSTAT1", 8);
  h.Q = c->Q;
  h.storage = c->storage;
  h.nx = c->nx;
  h.ny = c->ny;
  h.nz = c->nz;
  h.t = c->t;
  h.kind_h = c->kind_h;
  char hdr[64];
  memset(hdr, 0, 64);
  memcpy(hdr, &h, sizeof h);
  CK(cudaMemcpyAsync(buf, hdr, 64, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync((char*)buf + 64, c->buf[c->cur], state_bytes_raw(c), cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return XLB_OK;
}

int xlb_state_set(xlb_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return XLB_ERR_ARG;
  if (c->tape_open) return fail(c, XLB_ERR_STATE, "a tape is open");
  if (bytes < 64 + state_bytes_raw(c)) return fail(c, XLB_ERR_ARG, "buffer too small");
  char hdr[64];
  CK(cudaMemcpy(hdr, buf, 64, cudaMemcpyDefault));
  StateHeader h;
  memcpy(&h, hdr, sizeof h);
  if (memcmp(h.magic, "XLBSTAT1", 8) != 0) return fail(c, XLB_ERR_ARG, "not a serialized xlb state");
  if (h.Q != c->Q || h.storage != c->storage || h.nx != c->nx || h.ny != c->ny || h.nz != c->nz)
    return fail(c, XLB_ERR_ARG, "state of a different lattice, size or storage");
  CK(cudaMemcpyAsync(c->buf[c->cur], (const char*)buf + 64, state_bytes_raw(c), cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->t = h.t;
  c->kind_h = h.kind_h ? 1 : 0;
  c->has_init = true;
  if (c->kind_h) return boundary_pass(c, nullptr, c->buf[c->cur]);  // ghosts of the restored state
  return XLB_OK;
}

int xlb_populations(xlb_ctx* c, void** ptr, int64_t* plane) {
  if (!c || !ptr || !plane) return XLB_ERR_ARG;
  *ptr = c->buf[c->cur];
  *plane = c->plane;
  return XLB_OK;
}

// ---------------------------------------------------------------------------
// reverse mode

// The tape memory (checkpoints, k tape slots, two FP32 adjoint buffers) is one
// arena that outlives xlb_tape_end, so repeated gradients do not allocate; it
// grows when a larger tape needs it and is freed by xlb_tape_release.
int xlb_tape_end(xlb_ctx* c) {
  if (!c) return XLB_ERR_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->ckpt.clear();
  c->slots.clear();
  c->abar[0] = c->abar[1] = nullptr;
  c->tape_open = false;
  c->seg_loaded = -1;
  c->adj_t = -1;
  return XLB_OK;
}

int xlb_tape_release(xlb_ctx* c) {
  if (!c) return XLB_ERR_ARG;
  xlb_tape_end(c);
  if (c->tape_arena) cudaFree(c->tape_arena);
  c->tape_arena = nullptr;
  c->tape_arena_bytes = 0;
  return XLB_OK;
}

int xlb_tape_begin(xlb_ctx* c, int64_t n_steps, int64_t k) {
  if (!c) return XLB_ERR_ARG;
  if (n_steps < 1 || k < 1) return fail(c, XLB_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
  if (c->t != 0 || c->kind_h || !c->has_init) return fail(c, XLB_ERR_STATE, "open a tape right after xlb_init");
  if (c->coll == XLB_COLL_KBC) return fail(c, XLB_ERR_UNSUPPORTED, "the adjoint covers BGK and NONE collisions");
  if (c->storage == XLB_STORE_BF16)
    return fail(c, XLB_ERR_UNSUPPORTED,
                "the adjoint covers FP32 and FP16 storage (with BF16 the gradient misses the 5e-3 storage bound)");
  if (c->has_inlet_outlet)
    return fail(c, XLB_ERR_UNSUPPORTED, "the adjoint does not cover inlet/outlet or full-way (FWALL) cells");
  xlb_tape_end(c);
  if (k > n_steps) k = n_steps;
  const int64_t n_ckpt = (n_steps - 1) / k;
  const size_t sb = (state_bytes_raw(c) + 255) / 256 * 256;
  const size_t ab = (sizeof(float) * state_elems(c) + 255) / 256 * 256;
  if ((uint64_t)(n_ckpt + k) > (SIZE_MAX - 2 * ab) / sb)
    return fail(c, XLB_ERR_OOM, "a tape of %lld states does not fit in memory", (long long)(n_ckpt + k));
  const size_t need = (size_t)(n_ckpt + k) * sb + 2 * ab;
  if (c->tape_arena_bytes < need) {
    if (c->tape_arena) cudaFree(c->tape_arena);
    c->tape_arena = nullptr;
    c->tape_arena_bytes = 0;
    cudaError_t e = cudaMalloc(&c->tape_arena, need);
    if (e != cudaSuccess) {
      c->tape_arena = nullptr;
      return cuda_fail(c, e, "cudaMalloc(tape)");
    }
    c->tape_arena_bytes = need;
  }
  char* p = c->tape_arena;
  for (int64_t s = 0; s < n_ckpt; ++s, p += sb) c->ckpt.push_back(p);
  for (int64_t j = 0; j < k; ++j, p += sb) c->slots.push_back(p);
  c->abar[0] = reinterpret_cast<float*>(p);
  c->abar[1] = reinterpret_cast<float*>(p + ab);
  c->tape_open = true;
  c->tape_T = n_steps;
  c->tape_k = k;
  return XLB_OK;
}

static int ensure_adjoint_buffers(xlb_ctx* c) { return c->tape_open ? XLB_OK : XLB_ERR_STATE; }

static AdjointArgs adjoint_args(xlb_ctx* c) {
  AdjointArgs a;
  memset(&a, 0, sizeof a);
  a.p = make_params(c);
  a.Q = c->Q;
  a.storage = c->storage;
  a.coll = c->coll;
  a.ucs = c->N;
  a.stream = c->stream;
  return a;
}

static int adispatch(xlb_ctx* c, AdjOp op, const AdjointArgs& a) {
  int r = launch_adjoint(op, a);
  if (r != 0) return fail(c, XLB_ERR_UNSUPPORTED, "adjoint launch %d rejected (code %d)", (int)op, r);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint kernel launch");
  return XLB_OK;
}

int xlb_adjoint_seed_macro(xlb_ctx* c, const float* drho, const float* du) {
  if (!c) return XLB_ERR_ARG;
  if (!c->tape_open) return fail(c, XLB_ERR_STATE, "no tape open");
  if (c->t != c->tape_T || !c->kind_h) return fail(c, XLB_ERR_STATE, "take all %lld taped steps first", (long long)c->tape_T);
  int r = ensure_adjoint_buffers(c);
  if (r) return r;
  const size_t n = (size_t)c->N;
  const float* dr = drho;
  const float* duu = du;
  if ((drho && !is_device_ptr(drho)) || (du && !is_device_ptr(du))) {
    r = ensure_stage(c, (1 + c->D) * n * sizeof(float));
    if (r) return r;
    if (drho) {
      CK(cudaMemcpyAsync(c->stage, drho, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
      dr = (const float*)c->stage;
    }
    if (du) {
      CK(cudaMemcpyAsync((float*)c->stage + n, du, (size_t)c->D * n * sizeof(float), cudaMemcpyHostToDevice,
                         c->stream));
      duu = (const float*)c->stage + n;
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  AdjointArgs a = adjoint_args(c);
  a.state = c->buf[c->cur];
  a.fields_in = dr;
  a.fields_in2 = duu;
  a.abar_out = c->abar[0];
  r = adispatch(c, ADJ_SEED, a);
  if (r) return r;
  c->acur = 0;
  c->adj_t = c->tape_T;
  return XLB_OK;
}

int xlb_adjoint_seed_kinetic_energy(xlb_ctx* c, const int64_t box_lo[3], const int64_t box_hi[3], double scale) {
  if (!c) return XLB_ERR_ARG;
  if (!c->tape_open) return fail(c, XLB_ERR_STATE, "no tape open");
  if (c->t != c->tape_T || !c->kind_h) return fail(c, XLB_ERR_STATE, "take all %lld taped steps first", (long long)c->tape_T);
  int r = check_box(c, box_lo, box_hi);
  if (r) return r;
  AdjointArgs a = adjoint_args(c);
  a.state = c->buf[c->cur];
  a.abar_out = c->abar[0];
  a.ke = 1;
  a.scale = (float)scale;
  for (int k = 0; k < 3; ++k) {
    a.box_lo[k] = (int)box_lo[k];
    a.box_hi[k] = (int)box_hi[k];
  }
  r = adispatch(c, ADJ_SEED, a);
  if (r) return r;
  c->acur = 0;
  c->adj_t = c->tape_T;
  return XLB_OK;
}

// Recompute the tape slots of segment s (states h_{sk+j-1}, j = 0..k-1; slot
// 0 of segment 0 is unused since h_{-1} does not exist).
static int load_segment(xlb_ctx* c, int64_t s) {
  if (c->seg_loaded == s) return XLB_OK;
  const int64_t k = c->tape_k;
  const int64_t jmax = std::min<int64_t>(k - 1, c->tape_T - 1 - s * k);
  int r;
  int64_t j0;
  if (s == 0) {
    if (jmax < 1) {
      c->seg_loaded = s;
      return XLB_OK;
    }
    r = launch_init(c, c->slots[1]);
    if (r) return r;
    r = launch_collide_local(c, c->slots[1]);
    if (r) return r;
    j0 = 2;
  } else {
    CK(cudaMemcpyAsync(c->slots[0], c->ckpt[s - 1], state_bytes_raw(c), cudaMemcpyDeviceToDevice, c->stream));
    j0 = 1;
  }
  for (int64_t j = j0; j <= jmax; ++j) {
    r = launch_step(c, c->slots[j - 1], c->slots[j]);
    if (r) return r;
  }
  c->seg_loaded = s;
  return XLB_OK;
}

int xlb_adjoint_step(xlb_ctx* c, int64_t n) {
  if (!c) return XLB_ERR_ARG;
  if (!c->tape_open || c->adj_t < 0) return fail(c, XLB_ERR_STATE, "seed the adjoint first");
  if (n < 0 || n > c->adj_t) return fail(c, XLB_ERR_ARG, "n must lie in [0, %lld]", (long long)c->adj_t);
  for (int64_t m = 0; m < n; ++m) {
    const int64_t t = c->adj_t - 1;  // produce fbar_t from fbar_{t+1}
    AdjointArgs a = adjoint_args(c);
    a.abar_in = c->abar[c->acur];
    a.abar_out = c->abar[c->acur ^ 1];
    int r;
    if (t >= 1) {
      const int64_t s = t / c->tape_k;
      r = load_segment(c, s);
      if (r) return r;
      a.state = c->slots[t - s * c->tape_k];
      cudaEvent_t* pe = prof_begin(c, 1);
      r = adispatch(c, ADJ_STEP, a);
      prof_end(c, pe);
    } else {
      a.fields_in = c->init_fields;
      a.fields_in2 = c->init_fields + c->N;
      r = adispatch(c, ADJ_STEP0, a);
    }
    if (r) return r;
    c->acur ^= 1;
    c->adj_t = t;
  }
  return XLB_OK;
}

int xlb_adjoint_init_grad(xlb_ctx* c, float* drho0, float* du0) {
  if (!c) return XLB_ERR_ARG;
  if (!c->tape_open || c->adj_t != 0) return fail(c, XLB_ERR_STATE, "run the adjoint back to step 0 first");
  if (!drho0 && !du0) return XLB_OK;
  const size_t n = (size_t)c->N;
  const bool host = !is_device_ptr(drho0 ? (void*)drho0 : (void*)du0);
  float* dr = drho0;
  float* du = du0;
  if (host) {
    int r = ensure_stage(c, (1 + c->D) * n * sizeof(float));
    if (r) return r;
    dr = drho0 ? (float*)c->stage : nullptr;
    du = du0 ? (float*)c->stage + n : nullptr;
  }
  AdjointArgs a = adjoint_args(c);
  a.abar_in = c->abar[c->acur];
  a.fields_in = c->init_fields;
  a.fields_in2 = c->init_fields + c->N;
  a.grad_rho = dr;
  a.grad_u = du;
  int r = adispatch(c, ADJ_INIT_GRAD, a);
  if (r) return r;
  if (host) {
    if (drho0) CK(cudaMemcpyAsync(drho0, dr, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (du0) CK(cudaMemcpyAsync(du0, du, (size_t)c->D * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return XLB_OK;
}

// ---------------------------------------------------------------------------
// profiling

int xlb_profile_enable(xlb_ctx* c, int on) {
  if (!c) return XLB_ERR_ARG;
  c->prof = on != 0;
  c->ev_used = 0;
  return XLB_OK;
}

int xlb_profile_read(xlb_ctx* c, int kernel, double* total_ms, int64_t* launches) {
  if (!c || !total_ms || !launches) return XLB_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  int64_t cnt = 0;
  for (size_t k = 0; k < c->ev_used; ++k) {
    if (c->ev_kind[k] != kernel) continue;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev_pool[k].a, c->ev_pool[k].b));
    tot += ms;
    ++cnt;
  }
  *total_ms = tot;
  *launches = cnt;
  c->ev_used = 0;
  return XLB_OK;
}

}  // extern "C"
