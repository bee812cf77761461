/*
 * xlb.h - C ABI of the GB300 lattice Boltzmann hot path (libxlb.so).
 *
 * The library advances a lattice Boltzmann simulation on one GPU: the fused
 * stream-and-collide update of Section 2 (Eqs. 1-2; BGK Eq. 3 with the
 * equilibrium of Eq. 5, or the KBC entropic collision Section 2 names), the
 * mask-driven boundary conditions of Section 3.5, the mixed storage precision
 * of Section 3.7, reverse-mode differentiation of the step (Section 3.6) and a
 * batched launch over many small 2D domains (the vmap batching of Section 6).
 *
 * Conventions shared by every call:
 *  - Every call returns an xlb_status; nothing aborts the process.
 *    xlb_last_error() gives a one-line reason for the last failure on a ctx.
 *  - Lattice fields are x-fastest: cell (x, y, z) sits at x + nx*(y + ny*z).
 *    Vector fields are component-major: u[a*N + cell], a = x, y (, z).
 *  - Pointers passed in may be host or device memory (the library asks CUDA
 *    which).  They are borrowed for the duration of the call only.
 *  - Work is queued on the ctx's stream.  Calls that read results into host
 *    memory synchronise that stream before returning; the others are
 *    asynchronous.
 *  - The library owns every population, mask, tape and scratch buffer.
 *  - Populations are stored as deviations f_i - w_i (rho0 = 1) in the chosen
 *    storage type; all arithmetic is FP32, global sums are FP64.
 */
#ifndef XLB_H
#define XLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xlb_ctx xlb_ctx;

typedef enum {
  XLB_OK = 0,
  XLB_ERR_ARG = 1,         /* invalid argument (null, size, code out of range)      */
  XLB_ERR_UNSUPPORTED = 2, /* valid but not provided (e.g. KBC on D3Q19)           */
  XLB_ERR_OOM = 3,         /* device allocation failed                              */
  XLB_ERR_CUDA = 4,        /* a CUDA call failed; xlb_last_error has its message   */
  XLB_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired                    */
  XLB_ERR_STATE = 6        /* call out of order (e.g. adjoint before a tape)       */
} xlb_status;

/* Lattices of Figure 1 (Section 3.2): the value is Q. */
enum { XLB_D2Q9 = 9, XLB_D3Q19 = 19, XLB_D3Q27 = 27 };

/* Collision models (Section 2): NONE streams only (a pure permutation). */
enum { XLB_COLL_NONE = 0, XLB_COLL_BGK = 1, XLB_COLL_KBC = 2 };

/* Storage precision of populations (Section 3.7 "compute/storage"): the
 * compute type is always FP32.  F16/BF16 store shifted populations
 * f_i - w_i (the centring Section 4.1 cites).  F16 rounds to nearest even.
 * BF16 rounds stochastically (up with probability equal to the discarded
 * fraction), from random bits hashed from the cell index and the cell's FP32
 * values, so that results are reproducible and identical in every kernel
 * variant; ghost values of boundary links round to nearest even. */
enum { XLB_STORE_F32 = 0, XLB_STORE_F16 = 1, XLB_STORE_BF16 = 2 };

/* Cell types of the mask (Section 3.5).  For a fluid-like or FWALL cell x
 * and a direction i whose source cell x - c_i is
 *   FLUID/INLET/OUTLET/FWALL: f_i(x) = h_i(x - c_i)           (Eq. 2, periodic)
 *   WALL:   f_i(x) = h_opp(i)(x)                                (halfway bounce-back)
 *   LID:    f_i(x) = h_opp(i)(x) + 2 w_i rho_w (c_i . u_w) / cs^2 (moving wall)
 *   EQ:     f_i(x) = f_i^eq(rho_w, u_w)                         (equilibrium BC)
 * where h is the post-collision state.  INLET cells then rebuild their c_x=+1
 * populations by Zou-He for the inlet velocity; OUTLET cells copy their
 * c_x=-1 populations from the cell at x-1 (zero-gradient outflow).  FWALL
 * cells are full-way bounce-back walls (the walls of the Section 5 cavity):
 * they stream like fluid cells, their collision is h_i = f_opp(i) (none under
 * XLB_COLL_NONE), they start at rest and report rho = 0, u = 0; the mass
 * they hold in transit is outside the fluid-cell sums of xlb_reduce. */
enum {
  XLB_CELL_FLUID = 0,
  XLB_CELL_WALL = 1,
  XLB_CELL_LID = 2,
  XLB_CELL_INLET = 3,
  XLB_CELL_OUTLET = 4,
  XLB_CELL_EQ = 5,
  XLB_CELL_FWALL = 6
};

/* ---- simulation context ------------------------------------------------ */

/* Create a simulation of nx*ny*nz cells (dims = {nx, ny, nz}; nz = 1 for
 * D2Q9) with relaxation rate omega = dt/tau (Eq. 3; tau from Eq. 4).
 * collision: XLB_COLL_*; KBC is defined on D2Q9 and D3Q27 only
 * (XLB_ERR_UNSUPPORTED on D3Q19).  storage: XLB_STORE_*.  cuda_stream: a
 * cudaStream_t to queue work on, or NULL for a stream the library creates.
 * Every face is periodic until a mask is set.  Allocates two population
 * buffers of Q*N elements.  A lattice holds at most 2^31 - 1 cells
 * (XLB_ERR_UNSUPPORTED beyond).  On failure *out is NULL. */
int xlb_create(xlb_ctx** out, int lattice, const int64_t dims[3], double omega, int collision, int storage,
               void* cuda_stream);

/* Release every buffer of the ctx (NULL is accepted). */
void xlb_destroy(xlb_ctx* ctx);

/* One-line description of the last failure on ctx ("" if none); valid until
 * the next call on ctx.  ctx may be NULL (reports creation failures). */
const char* xlb_last_error(const xlb_ctx* ctx);

/* Static name of a status code. */
const char* xlb_status_string(int status);

/* The velocity set of a lattice in the library's direction order (Figure 1,
 * rest velocity first), the order every direction index of this API uses:
 * c receives 3*Q ints (c_x, c_y, c_z per direction; c_z = 0 on D2Q9) and w,
 * if not NULL, the Q weights.  Host memory; XLB_ERR_ARG for a lattice other
 * than 9, 19, 27.  Needs no GPU. */
int xlb_lattice_table(int lattice, int32_t* c, double* w);

/* omega = 1 / (nu / cs^2 + 1/2) with dt = 1 (Eq. 4). */
double xlb_omega_from_nu(double nu);

/* Set the per-cell type mask (uint8 codes XLB_CELL_*, N cells, x fastest).
 * Codes >= 7 give XLB_ERR_ARG and leave the previous mask in place.  Between
 * steps, a new mask (like new boundary values from xlb_set_bc) acts from the
 * next step on: the current state keeps the boundaries it was streamed with.
 * XLB_ERR_STATE while a tape is open. */
int xlb_set_mask(xlb_ctx* ctx, const uint8_t* mask);

/* Sizes of the boundary tables of the current mask.  Whole face planes that
 * the mask fills with one boundary type are handled by coordinates and need
 * no table (with 16-bit storage the WALL / LID / EQ planes x = 0 and
 * x = nx - 1 are served by the table instead).  Whole INLET planes at x = 0
 * and OUTLET planes at x = nx - 1 (apart from cells on y / z faces) are
 * updated by the bulk pass; their cells then count as link owners, not as
 * fix-up cells.
 * n_links = number of (cell, direction) pairs, over FLUID cells, FWALL
 * cells of FWALL face planes and the cells of those inlet / outlet planes,
 * whose source cell is WALL, LID or EQ off the face planes; n_fix = number
 * of the other INLET and OUTLET cells plus the FWALL cells off the face
 * planes.  After each update a boundary pass writes, for every link, the
 * value the rule prescribes into the source cell's slot for that direction
 * (a ghost value, so the next update can pull every cell as if periodic)
 * and stores the fix-up cells, recomputed beside the bulk pass. */
int xlb_boundary_links(const xlb_ctx* ctx, int64_t* n_links, int64_t* n_fix);

/* Zou-He inlet velocity per cell (a velocity profile, e.g. the Poiseuille
 * inflow of the Section 4.3 cylinder): u holds D*N floats, component-major
 * (u_x of every cell, then u_y, ...; host or device memory, copied); only the
 * entries of INLET cells are used.  NULL returns to the constant velocity of
 * xlb_set_bc(XLB_CELL_INLET).  Acts from the next step on.  XLB_ERR_STATE
 * while a tape is open. */
int xlb_set_inlet_profile(xlb_ctx* ctx, const float* u);

/* Rule of the INLET cells (Section 4.3 names both): XLB_INLET_ZOU_HE (the
 * default; non-equilibrium bounce-back of each unknown c_x = +1 population:
 * f_i = f_opp(i) + f_i^eq - f_opp(i)^eq with rho from the known populations)
 * or XLB_INLET_REGULARIZED (Latt et al. 2008: the same rho; the unknown
 * populations' non-equilibrium parts by bounce-back; then every population is
 * rebuilt as f_i^eq(rho, u) + w_i / (2 cs^4) (c_i c_i - cs^2 I) : Pi^neq).
 * Acts from the next step on; XLB_ERR_ARG for an unknown scheme,
 * XLB_ERR_STATE while a tape is open. */
enum { XLB_INLET_ZOU_HE = 0, XLB_INLET_REGULARIZED = 1 };
int xlb_set_inlet_scheme(xlb_ctx* ctx, int scheme);

/* Inward normal n = sign e_axis (axis 0 = x, 1 = y, 2 = z; sign +1 or -1)
 * of the boundary the INLET cells lie on; (0, +1), an inflow along +x, by
 * default.  INLET cells are velocity boundaries: the unknown populations are
 * those entering the fluid through the boundary (c_i . n = +1), rho comes
 * from the known ones, [sum_{c.n=0} f_i + 2 sum_{c.n=-1} f_i] / (1 - u.n), and
 * the rule of xlb_set_inlet_scheme rebuilds them.  With a velocity parallel
 * to the wall (e.g. normal (2, -1) on the top plane and u = (U, 0, 0)) the
 * regularized rule is the regularized moving wall Section 4.2 uses for its
 * lid.  Acts from the next step on; XLB_ERR_ARG for an axis beyond the
 * lattice's dimension or another sign, XLB_ERR_STATE while a tape is open. */
int xlb_set_inlet_normal(xlb_ctx* ctx, int axis, int sign);

/* Curved no-slip walls: Bouzidi's linear interpolated bounce-back (Bouzidi,
 * Firdaouss and Lallemand 2001, named in Section 4.3) on listed links.
 * Link k joins FLUID cell cell[k] (index x + nx*(y + ny*z)) to its WALL
 * neighbour cell[k] + c_dir[k] (dir[k] in 1..Q-1, Figure 1 order); the wall
 * crosses the link at the fraction q[k] in [0, 1] of its length from the
 * fluid cell.  With h the post-collision state and j = opp(dir[k]) the
 * direction the fluid cell then pulls from the wall cell:
 *   q <  1/2: f_j(x) = 2q h_i(x) + (1 - 2q) h_i(x + c_j), i = dir[k]
 *             (h_i(x) if x + c_j is not FLUID),
 *   q >= 1/2: f_j(x) = h_i(x) / (2q) + (2q - 1) / (2q) h_j(x).
 * Unlisted WALL links keep halfway bounce-back (q = 1/2).  Arrays are host
 * memory; the list replaces any earlier one (n = 0 clears it) and acts from
 * the next step on; a new mask clears it.  XLB_ERR_ARG (nothing changed) if
 * a link is not a ghost link of the mask (the cell is not FLUID, the
 * neighbour is not WALL, or the neighbour lies on a boundary face plane) or
 * a q is outside [0, 1]; XLB_ERR_STATE before a mask or while a tape is open. */
int xlb_set_wall_distances(xlb_ctx* ctx, int64_t n, const int64_t* cell, const int32_t* dir, const float* q);

/* Momentum-exchange force on the WALL cells off the boundary faces (Mei et
 * al. 2002 as Caiazzo and Junk 2008 apply it to interpolated walls; the lift
 * and drag of Section 4.3) in the most recent update, from step t-1 to the
 * current step t: the sum over the ghost links (FLUID cell x, WALL cell
 * x + c_i) of c_i [h_i(x, t-1) + f_opp(i)(x, t)], with h the post-collision
 * populations of step t-1 and f the post-stream populations of step t,
 * summed in FP64.  out receives 3 doubles (F_z = 0 on D2Q9); a device pointer is
 * written asynchronously on the ctx stream (for a time series without host
 * round trips), a host pointer synchronously.  Links of INLET / OUTLET /
 * FWALL cells and walls on the boundary faces are not included.
 * XLB_ERR_STATE before the first step after xlb_init (or after a change of
 * mask or boundary values, until the next step). */
int xlb_wall_force(xlb_ctx* ctx, double* out);

/* Prescribed state of a boundary type: XLB_CELL_LID (rho_w, u_w of the
 * moving wall), XLB_CELL_INLET (Zou-He velocity u; rho ignored) or
 * XLB_CELL_EQ (rho_w, u_w of the equilibrium BC).  u has 3 components (the
 * third is ignored on D2Q9).  Default: rho = 1, u = 0. */
int xlb_set_bc(xlb_ctx* ctx, int cell_type, float rho, const float u[3]);

/* Constant body force F (3 components) on fluid-like cells, applied by the
 * exact-difference method (Section 6.1): f* += f^eq(rho, u + F/rho) - f^eq(rho, u).
 * The reported velocity becomes (j + F/2) / rho. */
int xlb_set_force(xlb_ctx* ctx, const float F[3]);

/* f_0 = f^eq(rho, u) (Eq. 5) on fluid-like cells, boundary values elsewhere;
 * resets the step counter to 0.  rho: N values or NULL (rho = 1); u: D*N
 * values, component-major, or NULL (u = 0).  The fields are kept on the
 * device for xlb_adjoint_init_grad. */
int xlb_init(xlb_ctx* ctx, const float* rho, const float* u);

/* Advance n >= 0 time steps: f_{t+1} = S_bc(C(f_t)) (Eqs. 1-2, Section 3.6).
 * Asynchronous.  While a tape is open (xlb_tape_begin) the checkpoints of the
 * tape are recorded and stepping past its length is XLB_ERR_STATE. */
int xlb_step(xlb_ctx* ctx, int64_t n);

/* Graph replay of the update (for small lattices, where launch overhead
 * dominates): with steps_per_graph = g >= 1, xlb_step advances in blocks of
 * g updates by launching a CUDA graph of them, captured on the ctx stream at
 * first use and captured again after any change of the mask, boundary
 * values, force or kernel variant; the first update after xlb_init and any
 * remainder of fewer than g updates are launched directly.  g = 0 (the
 * default) launches every update.  Results are identical either way.  The
 * capture needs the ctx stream idle and not capturing, with no other thread
 * queuing work on it during xlb_step; graphs are not used while a tape is
 * open or profiling is on.  XLB_ERR_ARG for g outside [0, 100000]. */
int xlb_set_step_graph(xlb_ctx* ctx, int64_t steps_per_graph);

/* Number of steps taken since xlb_init / xlb_state_set. */
int xlb_get_time(const xlb_ctx* ctx, int64_t* t);

/* rho (N values) and u (D*N, component-major) of the current post-stream
 * state (Eqs. 6-7).  Either pointer may be NULL.  Solid cells report zeros;
 * EQ cells report their prescribed state. */
int xlb_macroscopic(xlb_ctx* ctx, float* rho, float* u);

/* FP64 totals over fluid-like cells of the current post-stream state:
 * out_mass[0] = sum rho, out_mom[0..2] = sum j (bare momentum, no force
 * shift).  Host outputs; synchronises. */
int xlb_reduce(xlb_ctx* ctx, double out_mass[1], double out_mom[3]);

/* FP64 kinetic energy L = sum over the box of (1/2) rho |u|^2 of the current
 * post-stream state's observables (those xlb_macroscopic returns: u is the
 * reported velocity (j + F/2) / rho, EQ cells count with their prescribed
 * state, solid cells with zero) -- the rollout loss of the differentiable
 * workloads (Section 6 takes gradients of such losses).  The box is
 * [box_lo[a], box_hi[a]) per axis (x, y, z; 0 <= lo < hi <= extent, z range
 * [0, 1) on D2Q9).  rho and u are formed in FP32, the squares and the sum in
 * FP64.  out: one double, device memory (written asynchronously on the ctx
 * stream) or host memory (synchronises). */
int xlb_kinetic_energy(xlb_ctx* ctx, const int64_t box_lo[3], const int64_t box_hi[3], double* out);

/* FP64 sum of squares of n floats in device memory (the squared norm of a
 * gradient), on the ctx stream; out as for xlb_kinetic_energy.  XLB_ERR_ARG
 * for host memory. */
int xlb_sum_squares(xlb_ctx* ctx, const float* x, int64_t n, double* out);

/* Wait for all work queued on the ctx's stream; XLB_ERR_TIMEOUT if a bounded
 * wait inside a kernel expired since the last check (the results of those
 * steps are invalid). */
int xlb_synchronize(xlb_ctx* ctx);

/* FP64 totals of stored populations without any device allocation.  The
 * paper has no counterpart.  It serves callers that cannot call cudaMalloc:
 * latency-critical loops (the allocator may synchronise the device and takes
 * unbounded time), host frameworks that own all device memory through their
 * own pools under a fixed budget, and recovery paths that run after the
 * device has run out of memory.  It reduces `populations` (device memory: Q
 * planes of plane_stride elements of the storage type, each holding
 * f_i - w_i for the N = nx*ny*nz cells, x fastest -- the layout
 * xlb_populations exposes) over the fluid-like cells of `mask` (device
 * memory, uint8 XLB_CELL_* codes; NULL = all cells): out[0] = sum rho,
 * out[1..3] = sum j, of the populations as stored.  After xlb_step the live
 * buffer holds the post-collision state (the next update streams it), not
 * the post-stream state xlb_reduce sums: the two totals agree on periodic
 * lattices without a body force and differ with walls, inlets or a moving
 * lid.  `out` is 4 doubles in device memory (written on the stream) or host
 * memory (the call then copies and synchronises the stream, and returns
 * XLB_ERR_ARG if the stream is being captured).  The partial sums live in
 * one fixed array of 128 KiB compiled into the library, which every GPU that
 * loads it keeps until the process exits: at most 67,108,864 cells (4096
 * partial sums of 16384 cells); larger lattices give XLB_ERR_ARG.  The first
 * call on a device looks up the array's address with that device current;
 * make that first call before capturing any stream.  Calls share the array:
 * calls that overlap on the GPU race, so order them on one stream.  Each call
 * rewrites every partial it reads, so nothing needs clearing between
 * calls. */
int xlb_moments_noalloc(int lattice, const int64_t dims[3], int storage, const void* populations,
                        int64_t plane_stride, const uint8_t* mask, double* out, void* cuda_stream);

/* ---- checkpoint / resume (Section 3.7) --------------------------------- */

/* Size in bytes of a serialized state (header + populations). */
int xlb_state_bytes(const xlb_ctx* ctx, size_t* bytes);

/* Serialize the state (step counter, whether it holds pre- or
 * post-collision populations, raw stored deviations) into buf (host or
 * device, at least xlb_state_bytes).  Synchronises. */
int xlb_state_get(xlb_ctx* ctx, void* buf, size_t bytes);

/* Restore a state written by xlb_state_get of a ctx with the same lattice,
 * dims and storage (XLB_ERR_ARG otherwise). */
int xlb_state_set(xlb_ctx* ctx, const void* buf, size_t bytes);

/* Device pointer and element stride of the live population buffer (for
 * zero-copy inspection; valid until the next xlb_step). */
int xlb_populations(xlb_ctx* ctx, void** dev_ptr, int64_t* plane_stride);

/* ---- reverse mode (Section 3.6 grad of step; Section 7 adjoint) -------- */

/* Open a tape right after xlb_init: the next xlb_step calls (n_steps in
 * total) record a checkpoint every checkpoint_every steps.  The adjoint then
 * recomputes each segment from its checkpoint.  BGK or NONE collision, FP32
 * or FP16 storage (the FP16 gradient is that of the FP16 forward, each
 * rounding taken as the identity); BF16 storage and masks with INLET /
 * OUTLET / FWALL cells are XLB_ERR_UNSUPPORTED. */
int xlb_tape_begin(xlb_ctx* ctx, int64_t n_steps, int64_t checkpoint_every);

/* Seed the adjoint at the final step with the loss cotangents of the
 * observables xlb_macroscopic returns: dL_drho (N) and dL_du (D*N); either
 * may be NULL (zero).  Requires all n_steps of the tape to have been taken. */
int xlb_adjoint_seed_macro(xlb_ctx* ctx, const float* dL_drho, const float* dL_du);

/* Seed the adjoint at the final step with scale times the cotangent of the
 * kinetic-energy loss of xlb_kinetic_energy over the same box, formed on the
 * GPU from the final state: dL/drho = |u|^2 / 2 and dL/du = rho u inside the
 * box, zero outside.  Same preconditions as xlb_adjoint_seed_macro. */
int xlb_adjoint_seed_kinetic_energy(xlb_ctx* ctx, const int64_t box_lo[3], const int64_t box_hi[3], double scale);

/* Propagate the adjoint n steps backwards (n <= steps remaining). */
int xlb_adjoint_step(xlb_ctx* ctx, int64_t n);

/* After the adjoint reached step 0: gradients of the loss with respect to
 * the initial fields given to xlb_init, dL_drho0 (N) and dL_du0 (D*N); either
 * may be NULL.  Solid and EQ cells get 0. */
int xlb_adjoint_init_grad(xlb_ctx* ctx, float* dL_drho0, float* dL_du0);

/* Close the tape.  Its memory (checkpoints, tape slots, adjoint buffers) is
 * kept for the next tape of the same or smaller size, so repeated gradients
 * allocate nothing after the first. */
int xlb_tape_end(xlb_ctx* ctx);

/* Close the tape and free its memory. */
int xlb_tape_release(xlb_ctx* ctx);

/* ---- kernel selection -------------------------------------------------- */

/* Variants of the bulk pass of an update (same arithmetic):
 *   XLB_KERNEL_DIRECT: one thread per cell, populations loaded straight from
 *     global memory;
 *   XLB_KERNEL_VEC:    4 consecutive cells per thread, one aligned 4-wide load
 *     per direction, the +-x neighbour element exchanged by warp shuffles
 *     (16-bit storage, D2Q9 / D3Q19, BGK, nx % 4 == 0);
 *   XLB_KERNEL_VEC2:   the same with 2 cells per thread and 32-bit words
 *     (nx even);
 *   XLB_KERNEL_AUTO:   the default: with FP16 storage VEC on lattices without
 *     boundary planes and VEC2 with them, else DIRECT (the fastest measured
 *     on 256^3 D3Q19 lattices; BF16 and FP32 run DIRECT).
 * A mask with an FWALL face plane always runs DIRECT. */
enum { XLB_KERNEL_AUTO = 0, XLB_KERNEL_DIRECT = 1, XLB_KERNEL_VEC = 2, XLB_KERNEL_VEC2 = 3 };

/* Choose the variant (XLB_ERR_UNSUPPORTED if it cannot run this ctx). */
int xlb_set_kernel(xlb_ctx* ctx, int variant);

/* The variant the next update launches (DIRECT, VEC or VEC2). */
int xlb_get_kernel(const xlb_ctx* ctx, int* variant);

/* ---- batched small 2D domains (Section 6 batching) --------------------- */

typedef struct xlb_batch xlb_batch;

/* n_domains independent D2Q9 BGK domains of nx[d] x ny[d] cells (each at
 * most 2^26 cells, all together at most 2^31 - 1), relaxation omega, storage
 * XLB_STORE_*.  Every domain is periodic in x and y unless its mask says
 * otherwise.  The library owns all buffers. */
int xlb_batch_create(xlb_batch** out, int n_domains, const int32_t* nx, const int32_t* ny, double omega,
                     int storage, void* cuda_stream);
void xlb_batch_destroy(xlb_batch* b);
const char* xlb_batch_last_error(const xlb_batch* b);

/* Cell masks (concatenated per domain, each x fastest; FLUID or WALL codes
 * only, XLB_ERR_UNSUPPORTED otherwise) and body forces (2 floats per domain,
 * exact-difference forcing); either may be NULL to keep the current one.
 * Host or device memory. */
int xlb_batch_set_masks(xlb_batch* b, const uint8_t* masks, const float* forces);

/* f_0 = f^eq(rho, u) per cell: rho (total cells) and u (2 per cell,
 * interleaved u_x, u_y) concatenated like the masks, or NULL (1 and 0). */
int xlb_batch_init(xlb_batch* b, const float* rho, const float* u);

/* Advance every domain n steps in one persistent launch: each CTA takes
 * domains from a queue, largest first, and runs all n steps of one domain
 * before the next.  The launch is captured in a CUDA graph on first use and
 * replayed while n and the launch shape stay the same. */
int xlb_batch_step(xlb_batch* b, int64_t n);

/* The same n steps with one ordinary launch per domain and step (the
 * baseline the persistent launch replaces). */
int xlb_batch_step_per_domain(xlb_batch* b, int64_t n);

/* Launch shape of xlb_batch_step: threads per CTA (32..1024, a multiple of
 * 32) and resident CTAs per SM (1..32, capped by occupancy). */
int xlb_batch_set_launch(xlb_batch* b, int threads, int ctas_per_sm);

/* Autotuner: time every candidate shape over sample_steps updates on a saved
 * copy of the state (restored afterwards), keep the fastest, append it to the
 * cache file (NULL: no cache; a matching line skips the timing). */
int xlb_batch_tune(xlb_batch* b, int sample_steps, const char* cache_path, int* best_threads, int* best_ctas);

/* rho (total cells) and u (2 per cell) of every domain's post-stream state;
 * reported u = (j + F/2) / rho; WALL cells 0.  Host or device; synchronises. */
int xlb_batch_macroscopic(xlb_batch* b, float* rho, float* u);

int xlb_batch_info(const xlb_batch* b, int64_t* total_cells, int64_t* t, int* threads, int* ctas_per_sm);
int xlb_batch_synchronize(xlb_batch* b);

/* ---- timing of the hot kernels ----------------------------------------- */

/* Total device time in ms of the launches of one kernel class recorded
 * since the last reset, measured with CUDA events on the ctx's stream, and
 * the number of launches.  kernel: 0 = fused stream-collide, 1 = adjoint step.
 * Enable with xlb_profile_enable(ctx, 1) (adds two event records per launch). */
int xlb_profile_enable(xlb_ctx* ctx, int on);
int xlb_profile_read(xlb_ctx* ctx, int kernel, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* XLB_H */
