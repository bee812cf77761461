"""Helpers shared by the GPU parity tests: run a case through the C ABI and
through the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

from oracle import lbm as O
from paper_2311_16080_gb300 import xlb as X

W = {q: O.Lattice(q).w for q in (9, 19, 27)}


def rel_l2(a, b, sel=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if sel is not None:
        a = a[..., sel]
        b = b[..., sel]
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


class Case:
    """One simulation set-up, runnable on the GPU and in the oracle."""

    def __init__(self, q, shape, omega, collision="bgk", mask=None, force=None, lid=None, inlet=None,
                 eq=None, rho0=None, u0=None, inlet_scheme="zou_he", inlet_normal=(0, 1)):
        self.q = q
        self.lat = O.Lattice(q)
        self.shape = tuple(shape)  # (ny, nx) or (nz, ny, nx)
        self.omega = omega
        self.collision = collision
        self.mask = mask if mask is not None else np.zeros(self.shape, np.uint8)
        self.force = force
        self.lid = lid      # (rho, u)
        self.inlet = inlet  # u
        self.eq = eq        # (rho, u)
        self.inlet_scheme = inlet_scheme
        self.inlet_normal = inlet_normal
        d = self.lat.d
        self.rho0 = rho0 if rho0 is not None else np.ones(self.shape)
        self.u0 = u0 if u0 is not None else np.zeros((d,) + self.shape)

    @property
    def dims(self):
        return tuple(reversed(self.shape))

    def params(self):
        d = self.lat.d
        bc = O.BC(d,
                  lid_u=self.lid[1][:d] if self.lid else None, lid_rho=self.lid[0] if self.lid else 1.0,
                  inlet_u=self.inlet[:d] if self.inlet else None,
                  eq_rho=self.eq[0] if self.eq else 1.0, eq_u=self.eq[1][:d] if self.eq else None,
                  inlet_scheme=self.inlet_scheme, inlet_normal=self.inlet_normal)
        return O.Params(self.lat, self.omega, collision=self.collision,
                        force=self.force[:d] if self.force else None, bc=bc)

    def oracle(self, steps):
        p = self.params()
        f = O.init_state(self.lat, self.rho0, self.u0, self.mask, p)
        f = O.run(self.lat, f, self.mask, p, steps)
        return O.macroscopic(self.lat, f, self.mask, p), f

    def gpu_sim(self, storage="f32", variant="auto"):
        sim = X.Simulation(self.q, self.dims, self.omega, self.collision, storage)
        sim.set_kernel(variant)
        if self.mask.any():
            sim.set_mask(np.ascontiguousarray(self.mask, dtype=np.uint8))
        if self.lid:
            sim.set_bc(X.XLB_CELL_LID, self.lid[0], self.lid[1])
        if self.inlet:
            sim.set_bc(X.XLB_CELL_INLET, 1.0, self.inlet)
        if self.inlet_scheme != "zou_he":
            sim.set_inlet_scheme(self.inlet_scheme)
        if tuple(self.inlet_normal) != (0, 1):
            sim.set_inlet_normal(*self.inlet_normal)
        if self.eq:
            sim.set_bc(X.XLB_CELL_EQ, self.eq[0], self.eq[1])
        if self.force:
            sim.set_force(self.force)
        sim.init(np.ascontiguousarray(self.rho0, dtype=np.float32),
                 np.ascontiguousarray(self.u0, dtype=np.float32))
        return sim

    def gpu(self, steps, storage="f32", variant="auto"):
        sim = self.gpu_sim(storage, variant)
        sim.step(steps)
        rho, u = sim.macroscopic()
        sim.close()
        return rho, u


def storage_dtype(storage):
    return {"f32": np.float32, "f16": np.float16, "bf16": np.uint16}[storage]


def bf16_to_f64(raw_u16):
    return (raw_u16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def raw_to_f64(raw, storage):
    if storage == "bf16":
        return bf16_to_f64(raw)
    return raw.astype(np.float64)


def f64_to_raw(v, storage):
    if storage == "bf16":
        b = v.astype(np.float32).view(np.uint32)
        assert np.all((b & 0xFFFF) == 0), "value not representable in bf16"
        return (b >> 16).astype(np.uint16)
    return v.astype(storage_dtype(storage))
