"""Thin Python binding of libxlb.so (include/xlb.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and raises
``XlbError`` on a non-zero status.  Buffers may be torch tensors (host or
CUDA; their ``data_ptr()`` is passed), numpy arrays or raw integer addresses.
Every step of the lattice Boltzmann path runs in the library's CUDA kernels;
if the library is missing, loading raises instead of falling back to any
CPU implementation.

``Simulation`` is a small convenience wrapper over one ctx, and
``KineticEnergyRollout()`` (the torch.autograd.Function class) / ``rollout``
expose the adjoint to torch autograd.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libxlb.so")

XLB_OK, XLB_ERR_ARG, XLB_ERR_UNSUPPORTED, XLB_ERR_OOM, XLB_ERR_CUDA, XLB_ERR_TIMEOUT, XLB_ERR_STATE = range(7)
XLB_D2Q9, XLB_D3Q19, XLB_D3Q27 = 9, 19, 27
XLB_COLL_NONE, XLB_COLL_BGK, XLB_COLL_KBC = 0, 1, 2
XLB_STORE_F32, XLB_STORE_F16, XLB_STORE_BF16 = 0, 1, 2
XLB_KERNEL_AUTO, XLB_KERNEL_DIRECT, XLB_KERNEL_VEC, XLB_KERNEL_VEC2 = 0, 1, 2, 3
XLB_CELL_FLUID, XLB_CELL_WALL, XLB_CELL_LID, XLB_CELL_INLET, XLB_CELL_OUTLET, XLB_CELL_EQ, XLB_CELL_FWALL = range(7)
XLB_INLET_ZOU_HE, XLB_INLET_REGULARIZED = 0, 1

STORAGE = {"f32": XLB_STORE_F32, "f16": XLB_STORE_F16, "bf16": XLB_STORE_BF16}
COLLISION = {"none": XLB_COLL_NONE, "bgk": XLB_COLL_BGK, "kbc": XLB_COLL_KBC}


class XlbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None

_vp, _i, _i64, _d, _f = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_float
_PROTOS = {
    "xlb_create": (_i, [C.POINTER(_vp), _i, C.POINTER(_i64), _d, _i, _i, _vp]),
    "xlb_destroy": (None, [_vp]),
    "xlb_last_error": (C.c_char_p, [_vp]),
    "xlb_status_string": (C.c_char_p, [_i]),
    "xlb_omega_from_nu": (_d, [_d]),
    "xlb_lattice_table": (_i, [_i, _vp, _vp]),
    "xlb_set_mask": (_i, [_vp, _vp]),
    "xlb_set_bc": (_i, [_vp, _i, _f, C.POINTER(_f)]),
    "xlb_boundary_links": (_i, [_vp, C.POINTER(_i64), C.POINTER(_i64)]),
    "xlb_set_force": (_i, [_vp, C.POINTER(_f)]),
    "xlb_init": (_i, [_vp, _vp, _vp]),
    "xlb_step": (_i, [_vp, _i64]),
    "xlb_get_time": (_i, [_vp, C.POINTER(_i64)]),
    "xlb_macroscopic": (_i, [_vp, _vp, _vp]),
    "xlb_reduce": (_i, [_vp, C.POINTER(_d), C.POINTER(_d)]),
    "xlb_synchronize": (_i, [_vp]),
    "xlb_kinetic_energy": (_i, [_vp, C.POINTER(_i64), C.POINTER(_i64), _vp]),
    "xlb_sum_squares": (_i, [_vp, _vp, _i64, _vp]),
    "xlb_adjoint_seed_kinetic_energy": (_i, [_vp, C.POINTER(_i64), C.POINTER(_i64), _d]),
    "xlb_moments_noalloc": (_i, [_i, C.POINTER(_i64), _i, _vp, _i64, _vp, _vp, _vp]),
    "xlb_state_bytes": (_i, [_vp, C.POINTER(C.c_size_t)]),
    "xlb_state_get": (_i, [_vp, _vp, C.c_size_t]),
    "xlb_state_set": (_i, [_vp, _vp, C.c_size_t]),
    "xlb_populations": (_i, [_vp, C.POINTER(_vp), C.POINTER(_i64)]),
    "xlb_tape_begin": (_i, [_vp, _i64, _i64]),
    "xlb_adjoint_seed_macro": (_i, [_vp, _vp, _vp]),
    "xlb_adjoint_step": (_i, [_vp, _i64]),
    "xlb_adjoint_init_grad": (_i, [_vp, _vp, _vp]),
    "xlb_tape_end": (_i, [_vp]),
    "xlb_tape_release": (_i, [_vp]),
    "xlb_set_kernel": (_i, [_vp, _i]),
    "xlb_set_step_graph": (_i, [_vp, _i64]),
    "xlb_set_inlet_profile": (_i, [_vp, _vp]),
    "xlb_set_inlet_scheme": (_i, [_vp, _i]),
    "xlb_set_inlet_normal": (_i, [_vp, _i, _i]),
    "xlb_set_wall_distances": (_i, [_vp, _i64, _vp, _vp, _vp]),
    "xlb_wall_force": (_i, [_vp, _vp]),
    "xlb_get_kernel": (_i, [_vp, C.POINTER(_i)]),
    "xlb_batch_create": (_i, [C.POINTER(_vp), _i, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _d, _i, _vp]),
    "xlb_batch_destroy": (None, [_vp]),
    "xlb_batch_last_error": (C.c_char_p, [_vp]),
    "xlb_batch_set_masks": (_i, [_vp, _vp, _vp]),
    "xlb_batch_init": (_i, [_vp, _vp, _vp]),
    "xlb_batch_step": (_i, [_vp, _i64]),
    "xlb_batch_step_per_domain": (_i, [_vp, _i64]),
    "xlb_batch_set_launch": (_i, [_vp, _i, _i]),
    "xlb_batch_tune": (_i, [_vp, _i, C.c_char_p, C.POINTER(_i), C.POINTER(_i)]),
    "xlb_batch_macroscopic": (_i, [_vp, _vp, _vp]),
    "xlb_batch_info": (_i, [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i), C.POINTER(_i)]),
    "xlb_batch_synchronize": (_i, [_vp]),
    "xlb_profile_enable": (_i, [_vp, _i]),
    "xlb_profile_read": (_i, [_vp, _i, C.POINTER(_d), C.POINTER(_i64)]),
}


def load(path=None):
    """Load libxlb.so (built in-tree by ``paper_2311_16080_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libxlb.so not found at {path}; build it with "
                           "`python -m paper_2311_16080_gb300.build` (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _status_name(s):
    try:
        return load().xlb_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _ptr(buf):
    """Address of a buffer: torch tensor, numpy array, int or None."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _check(status, ctx=None):
    if status != XLB_OK:
        msg = load().xlb_last_error(ctx).decode(errors="replace")
        raise XlbError(status, msg)


def _vec3(v):
    v = list(v) + [0.0] * (3 - len(v))
    return (C.c_float * 3)(*[float(x) for x in v[:3]])


# ---- one wrapper per C entry point ------------------------------------------

def xlb_create(lattice, dims, omega, collision=XLB_COLL_BGK, storage=XLB_STORE_F32, cuda_stream=None):
    lib = load()
    out = C.c_void_p()
    d = list(dims) + [1] * (3 - len(dims))
    arr = (C.c_int64 * 3)(*[int(x) for x in d])
    _check(lib.xlb_create(C.byref(out), int(lattice), arr, float(omega), int(collision), int(storage),
                          cuda_stream))
    return out.value


def xlb_destroy(ctx):
    load().xlb_destroy(ctx)


def xlb_last_error(ctx=None):
    return load().xlb_last_error(ctx).decode()


def xlb_status_string(status):
    return load().xlb_status_string(int(status)).decode()


def xlb_omega_from_nu(nu):
    return load().xlb_omega_from_nu(float(nu))


def xlb_set_mask(ctx, mask):
    _check(load().xlb_set_mask(ctx, _ptr(mask)), ctx)


def xlb_boundary_links(ctx):
    nl, nf = C.c_int64(), C.c_int64()
    _check(load().xlb_boundary_links(ctx, C.byref(nl), C.byref(nf)), ctx)
    return nl.value, nf.value


def xlb_set_bc(ctx, cell_type, rho, u):
    _check(load().xlb_set_bc(ctx, int(cell_type), float(rho), _vec3(u)), ctx)


def xlb_set_force(ctx, F):
    _check(load().xlb_set_force(ctx, _vec3(F)), ctx)


def xlb_init(ctx, rho=None, u=None):
    _check(load().xlb_init(ctx, _ptr(rho), _ptr(u)), ctx)


def xlb_step(ctx, n):
    _check(load().xlb_step(ctx, int(n)), ctx)


def xlb_get_time(ctx):
    t = C.c_int64()
    _check(load().xlb_get_time(ctx, C.byref(t)), ctx)
    return t.value


def xlb_macroscopic(ctx, rho=None, u=None):
    _check(load().xlb_macroscopic(ctx, _ptr(rho), _ptr(u)), ctx)


def xlb_reduce(ctx):
    m = (C.c_double * 1)()
    j = (C.c_double * 3)()
    _check(load().xlb_reduce(ctx, m, j), ctx)
    return m[0], [j[0], j[1], j[2]]


def xlb_synchronize(ctx):
    _check(load().xlb_synchronize(ctx), ctx)


def _box(box, dims):
    """(lo[3], hi[3]) ctypes arrays from a box given as slices in the library
    field layout ([z, y, x] or [y, x]) or as ((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z))."""
    if isinstance(box, tuple) and box and isinstance(box[0], slice):
        sl = list(reversed(box)) + [slice(0, 1)] * (3 - len(box))
        lo = [s.start or 0 for s in sl]
        hi = [s.stop if s.stop is not None else dims[a] for a, s in enumerate(sl)]
    else:
        lo, hi = list(box[0]), list(box[1])
        lo += [0] * (3 - len(lo))
        hi += [1] * (3 - len(hi))
    return (C.c_int64 * 3)(*[int(v) for v in lo]), (C.c_int64 * 3)(*[int(v) for v in hi])


def xlb_kinetic_energy(ctx, box, dims, out=None):
    """FP64 sum over the box of (1/2) rho |u|^2 of the current observables.
    ``out``: None (returns a float), a 1-element float64 CUDA tensor (written
    asynchronously) or a host buffer."""
    lo, hi = _box(box, dims)
    if out is None:
        h = np.zeros(1, np.float64)
        _check(load().xlb_kinetic_energy(ctx, lo, hi, h.ctypes.data), ctx)
        return float(h[0])
    _check(load().xlb_kinetic_energy(ctx, lo, hi, _ptr(out)), ctx)
    return out


def xlb_sum_squares(ctx, x, n=None, out=None):
    """FP64 sum of squares of a float32 device buffer (returns a float, or
    writes a 1-element float64 buffer ``out``)."""
    if n is None:
        n = x.size if isinstance(x, np.ndarray) else x.numel()
    if out is None:
        h = np.zeros(1, np.float64)
        _check(load().xlb_sum_squares(ctx, _ptr(x), int(n), h.ctypes.data), ctx)
        return float(h[0])
    _check(load().xlb_sum_squares(ctx, _ptr(x), int(n), _ptr(out)), ctx)
    return out


def xlb_adjoint_seed_kinetic_energy(ctx, box, dims, scale=1.0):
    lo, hi = _box(box, dims)
    _check(load().xlb_adjoint_seed_kinetic_energy(ctx, lo, hi, float(scale)), ctx)


def xlb_moments_noalloc(lattice, dims, storage, populations, plane_stride, mask, out, cuda_stream=None):
    """FP64 (mass, j_x, j_y, j_z) of stored populations, allocating nothing
    (the library's fixed scratch array); ``out`` holds 4 doubles (host or
    device)."""
    d = list(dims) + [1] * (3 - len(dims))
    arr = (C.c_int64 * 3)(*[int(x) for x in d])
    s = load().xlb_moments_noalloc(int(lattice), arr, int(storage), _ptr(populations), int(plane_stride),
                                   _ptr(mask), _ptr(out), cuda_stream)
    if s != XLB_OK:
        raise XlbError(s, "xlb_moments_noalloc rejected its arguments or a CUDA call failed")


def xlb_state_bytes(ctx):
    n = C.c_size_t()
    _check(load().xlb_state_bytes(ctx, C.byref(n)), ctx)
    return n.value


def xlb_state_get(ctx, buf=None):
    if buf is None:
        buf = np.empty(xlb_state_bytes(ctx), dtype=np.uint8)
    nbytes = buf.nbytes if hasattr(buf, "nbytes") else buf.numel() * buf.element_size()
    _check(load().xlb_state_get(ctx, _ptr(buf), nbytes), ctx)
    return buf


def xlb_state_set(ctx, buf):
    nbytes = buf.nbytes if hasattr(buf, "nbytes") else buf.numel() * buf.element_size()
    _check(load().xlb_state_set(ctx, _ptr(buf), nbytes), ctx)


def xlb_populations(ctx):
    p = C.c_void_p()
    s = C.c_int64()
    _check(load().xlb_populations(ctx, C.byref(p), C.byref(s)), ctx)
    return p.value, s.value


def xlb_tape_begin(ctx, n_steps, checkpoint_every):
    _check(load().xlb_tape_begin(ctx, int(n_steps), int(checkpoint_every)), ctx)


def xlb_adjoint_seed_macro(ctx, dL_drho=None, dL_du=None):
    _check(load().xlb_adjoint_seed_macro(ctx, _ptr(dL_drho), _ptr(dL_du)), ctx)


def xlb_adjoint_step(ctx, n):
    _check(load().xlb_adjoint_step(ctx, int(n)), ctx)


def xlb_adjoint_init_grad(ctx, dL_drho0=None, dL_du0=None):
    _check(load().xlb_adjoint_init_grad(ctx, _ptr(dL_drho0), _ptr(dL_du0)), ctx)


def xlb_tape_end(ctx):
    _check(load().xlb_tape_end(ctx), ctx)


def xlb_tape_release(ctx):
    _check(load().xlb_tape_release(ctx), ctx)


def xlb_set_kernel(ctx, variant=XLB_KERNEL_AUTO):
    _check(load().xlb_set_kernel(ctx, int(variant)), ctx)


def xlb_lattice_table(lattice):
    """(c[Q, 3] int32, w[Q] float64): the library's velocity set and weights."""
    q = int(lattice)
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    _check(load().xlb_lattice_table(q, c.ctypes.data, w.ctypes.data))
    return c, w


def xlb_set_step_graph(ctx, steps_per_graph):
    _check(load().xlb_set_step_graph(ctx, int(steps_per_graph)), ctx)


def xlb_set_inlet_profile(ctx, u):
    """u: D*N float32 (numpy, torch tensor or raw pointer), or None."""
    if isinstance(u, np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float32)
    _check(load().xlb_set_inlet_profile(ctx, _ptr(u)), ctx)


def xlb_set_inlet_scheme(ctx, scheme):
    v = {"zou_he": XLB_INLET_ZOU_HE, "regularized": XLB_INLET_REGULARIZED}.get(scheme, scheme)
    _check(load().xlb_set_inlet_scheme(ctx, int(v)), ctx)


def xlb_set_inlet_normal(ctx, axis, sign):
    _check(load().xlb_set_inlet_normal(ctx, int(axis), int(sign)), ctx)


def xlb_set_wall_distances(ctx, cells, dirs, q):
    """Bouzidi wall distances of links (cell, direction toward the WALL
    neighbour, q in [0, 1]); host arrays."""
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    dirs = np.ascontiguousarray(dirs, dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    if not (cells.shape == dirs.shape == q.shape and cells.ndim == 1):
        raise ValueError("cells, dirs and q must be 1-D arrays of one length")
    _check(load().xlb_set_wall_distances(ctx, cells.size, cells.ctypes.data, dirs.ctypes.data,
                                         q.ctypes.data), ctx)


def xlb_wall_force(ctx, out=None):
    """Momentum-exchange force on the WALL cells (3 doubles).  With `out`
    (a device pointer or a torch CUDA tensor view) the result is written
    there asynchronously; otherwise it is returned as a numpy array."""
    if out is not None:
        p = out if isinstance(out, int) else out.data_ptr()
        _check(load().xlb_wall_force(ctx, C.c_void_p(p)), ctx)
        return None
    h = np.zeros(3, np.float64)
    _check(load().xlb_wall_force(ctx, h.ctypes.data), ctx)
    return h


def xlb_get_kernel(ctx):
    v = C.c_int()
    _check(load().xlb_get_kernel(ctx, C.byref(v)), ctx)
    return v.value


def xlb_profile_enable(ctx, on=True):
    _check(load().xlb_profile_enable(ctx, int(bool(on))), ctx)


def xlb_profile_read(ctx, kernel=0):
    ms = C.c_double()
    n = C.c_int64()
    _check(load().xlb_profile_read(ctx, int(kernel), C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def _bcheck(status, b):
    if status != XLB_OK:
        raise XlbError(status, load().xlb_batch_last_error(b).decode(errors="replace"))


def xlb_batch_create(nx, ny, omega, storage=XLB_STORE_F32, cuda_stream=None):
    out = C.c_void_p()
    n = len(nx)
    ax = (C.c_int32 * n)(*[int(v) for v in nx])
    ay = (C.c_int32 * n)(*[int(v) for v in ny])
    _bcheck(load().xlb_batch_create(C.byref(out), n, ax, ay, float(omega), int(storage), cuda_stream), None)
    return out.value


def xlb_batch_destroy(b):
    load().xlb_batch_destroy(b)


def xlb_batch_set_masks(b, masks=None, forces=None):
    _bcheck(load().xlb_batch_set_masks(b, _ptr(masks), _ptr(forces)), b)


def xlb_batch_init(b, rho=None, u=None):
    _bcheck(load().xlb_batch_init(b, _ptr(rho), _ptr(u)), b)


def xlb_batch_step(b, n):
    _bcheck(load().xlb_batch_step(b, int(n)), b)


def xlb_batch_step_per_domain(b, n):
    _bcheck(load().xlb_batch_step_per_domain(b, int(n)), b)


def xlb_batch_set_launch(b, threads, ctas_per_sm):
    _bcheck(load().xlb_batch_set_launch(b, int(threads), int(ctas_per_sm)), b)


def xlb_batch_tune(b, sample_steps, cache_path=None):
    t, c = C.c_int(), C.c_int()
    path = cache_path.encode() if cache_path else None
    _bcheck(load().xlb_batch_tune(b, int(sample_steps), path, C.byref(t), C.byref(c)), b)
    return t.value, c.value


def xlb_batch_macroscopic(b, rho, u):
    _bcheck(load().xlb_batch_macroscopic(b, _ptr(rho), _ptr(u)), b)


def xlb_batch_info(b):
    n, t, th, ct = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
    _bcheck(load().xlb_batch_info(b, C.byref(n), C.byref(t), C.byref(th), C.byref(ct)), b)
    return {"cells": n.value, "time": t.value, "threads": th.value, "ctas_per_sm": ct.value}


def xlb_batch_synchronize(b):
    _bcheck(load().xlb_batch_synchronize(b), b)


# ---- convenience wrapper -------------------------------------------------------

class Simulation:
    """One simulation context.  Fields use the library layout: scalars
    ``[nz, ny, nx]`` (or ``[ny, nx]``), vectors ``[D, ...]``."""

    def __init__(self, lattice, dims, omega, collision="bgk", storage="f32", stream=None):
        self.Q = int(lattice)
        self.D = 2 if self.Q == 9 else 3
        self.dims = tuple(int(x) for x in dims) + (1,) * (3 - len(dims))
        self.shape = (self.dims[1], self.dims[0]) if self.D == 2 else (self.dims[2], self.dims[1], self.dims[0])
        self.N = int(np.prod(self.shape))
        self.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.ctx = xlb_create(self.Q, self.dims, omega, self.collision, self.storage, stream)

    def close(self):
        if self.ctx:
            xlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mask(self, mask):
        xlb_set_mask(self.ctx, mask)

    def set_bc(self, cell_type, rho=1.0, u=(0.0, 0.0, 0.0)):
        xlb_set_bc(self.ctx, cell_type, rho, u)

    def set_force(self, F):
        xlb_set_force(self.ctx, F)

    def set_kernel(self, variant="auto"):
        v = {"auto": XLB_KERNEL_AUTO, "direct": XLB_KERNEL_DIRECT, "vec": XLB_KERNEL_VEC,
             "vec2": XLB_KERNEL_VEC2}.get(variant, variant)
        xlb_set_kernel(self.ctx, v)

    def kernel(self):
        return xlb_get_kernel(self.ctx)

    def set_step_graph(self, steps_per_graph):
        xlb_set_step_graph(self.ctx, steps_per_graph)

    def set_inlet_profile(self, u):
        xlb_set_inlet_profile(self.ctx, u)

    def set_inlet_scheme(self, scheme):
        xlb_set_inlet_scheme(self.ctx, scheme)

    def set_inlet_normal(self, axis, sign):
        xlb_set_inlet_normal(self.ctx, axis, sign)

    def set_wall_distances(self, cells, dirs, q):
        xlb_set_wall_distances(self.ctx, cells, dirs, q)

    def wall_force(self, out=None):
        return xlb_wall_force(self.ctx, out)

    def init(self, rho=None, u=None):
        xlb_init(self.ctx, rho, u)

    def step(self, n=1):
        xlb_step(self.ctx, n)

    @property
    def time(self):
        return xlb_get_time(self.ctx)

    def macroscopic(self, rho=None, u=None):
        """Fill (or allocate as numpy float32) rho [shape] and u [D, shape]."""
        if rho is None:
            rho = np.empty(self.shape, np.float32)
        if u is None:
            u = np.empty((self.D,) + self.shape, np.float32)
        xlb_macroscopic(self.ctx, rho, u)
        return rho, u

    def reduce(self):
        return xlb_reduce(self.ctx)

    def synchronize(self):
        xlb_synchronize(self.ctx)

    def state_get(self):
        return xlb_state_get(self.ctx)

    def state_set(self, buf):
        xlb_state_set(self.ctx, buf)

    def populations(self):
        """(raw host copy of the stored deviations as [Q, shape] in the storage
        dtype, kind_h) from a state snapshot."""
        buf = self.state_get()
        kind_h = int(np.frombuffer(buf[:64].tobytes(), dtype=np.int32)[12])
        dt = {0: np.float32, 1: np.float16, 2: np.uint16}[self.storage]
        raw = np.frombuffer(buf[64:].tobytes(), dtype=dt)
        align = 256 // raw.itemsize
        plane = (self.N + align - 1) // align * align
        return raw.reshape(self.Q, plane)[:, :self.N].reshape((self.Q,) + self.shape), kind_h


def _autograd_function():
    import torch

    class KineticEnergyRollout(torch.autograd.Function):
        """L(rho0[, u0]) = kinetic energy in a box after n steps from
        f_0 = f^eq(rho0, u0), differentiable through the library's adjoint.

        forward: xlb_init, xlb_tape_begin(n, k), xlb_step(n), xlb_kinetic_energy
        (FP64, on the device).  backward: xlb_adjoint_seed_kinetic_energy
        (scaled by the incoming cotangent), xlb_adjoint_step(n),
        xlb_adjoint_init_grad, xlb_tape_end.  rho0 / u0 are CUDA float32
        tensors in the library layout; the simulation's tape stays open from
        forward to backward."""

        @staticmethod
        def forward(ctx, rho0, u0, sim, n_steps, checkpoint_every, box):
            rho0 = rho0.detach().contiguous()
            u0 = None if u0 is None else u0.detach().contiguous()
            xlb_init(sim.ctx, rho0, u0)
            xlb_tape_begin(sim.ctx, n_steps, checkpoint_every)
            xlb_step(sim.ctx, n_steps)
            loss = torch.empty((), dtype=torch.float64, device=rho0.device)
            xlb_kinetic_energy(sim.ctx, box, sim.dims, loss)
            ctx.sim, ctx.n, ctx.box = sim, n_steps, box
            ctx.has_u0 = u0 is not None
            ctx.shape = tuple(rho0.shape)
            return loss

        @staticmethod
        def backward(ctx, g_out):
            sim = ctx.sim
            xlb_adjoint_seed_kinetic_energy(sim.ctx, ctx.box, sim.dims, float(g_out))
            xlb_adjoint_step(sim.ctx, ctx.n)
            g_rho = torch.empty(ctx.shape, dtype=torch.float32, device=g_out.device)
            g_u = (torch.empty((sim.D,) + ctx.shape, dtype=torch.float32, device=g_out.device)
                   if ctx.has_u0 else None)
            xlb_adjoint_init_grad(sim.ctx, g_rho, g_u)
            xlb_tape_end(sim.ctx)
            return g_rho, g_u, None, None, None, None

    return KineticEnergyRollout


_KER = None


def KineticEnergyRollout():
    """The torch.autograd.Function class of the kinetic-energy rollout."""
    global _KER
    if _KER is None:
        _KER = _autograd_function()
    return _KER


def rollout(sim, rho0, n_steps, checkpoint_every, box, u0=None):
    """Kinetic energy in ``box`` (slices in the field layout, or ((lo), (hi))
    in x, y, z) after ``n_steps`` of ``sim`` from f^eq(rho0, u0), as a
    differentiable FP64 torch scalar (the gradient runs the adjoint)."""
    return KineticEnergyRollout().apply(rho0, u0, sim, n_steps, checkpoint_every, box)


class Batch:
    """Many independent D2Q9 domains (dicts with nx, ny, mask[ny, nx] and
    force (Fx, Fy), as ``inputs.batched_channels`` builds them)."""

    def __init__(self, domains, omega, storage="f32", stream=None):
        self.domains = domains
        self.nx = [d["nx"] for d in domains]
        self.ny = [d["ny"] for d in domains]
        self.cells = [a * b for a, b in zip(self.nx, self.ny)]
        self.b = xlb_batch_create(self.nx, self.ny, omega, STORAGE.get(storage, storage), stream)

    def close(self):
        if self.b:
            xlb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_masks(self):
        masks = np.concatenate([np.ascontiguousarray(d["mask"], np.uint8).reshape(-1) for d in self.domains])
        forces = np.array([d.get("force", (0.0, 0.0)) for d in self.domains], np.float32).reshape(-1)
        xlb_batch_set_masks(self.b, masks, forces)

    def init(self, rho=None, u=None):
        xlb_batch_init(self.b, rho, u)

    def step(self, n):
        xlb_batch_step(self.b, n)

    def step_per_domain(self, n):
        xlb_batch_step_per_domain(self.b, n)

    def tune(self, sample_steps=20, cache_path=None):
        return xlb_batch_tune(self.b, sample_steps, cache_path)

    def macroscopic(self):
        """Per domain (rho[ny, nx], u[2, ny, nx]) as numpy arrays."""
        tot = sum(self.cells)
        rho = np.empty(tot, np.float32)
        u = np.empty(2 * tot, np.float32)
        xlb_batch_macroscopic(self.b, rho, u)
        out, o = [], 0
        for nx, ny, c in zip(self.nx, self.ny, self.cells):
            r = rho[o:o + c].reshape(ny, nx)
            uu = u[2 * o:2 * (o + c)].reshape(ny, nx, 2).transpose(2, 0, 1)
            out.append((r, uu))
            o += c
        return out
