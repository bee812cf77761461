"""Curved walls, lift and drag (Section 4.3): Bouzidi interpolated
bounce-back on listed links, a per-cell Zou-He inflow profile and the
momentum-exchange wall force, against the FP64 oracle on small cases of the
Schafer-Turek cylinder and on a D3Q19 sphere.

Bars: FP32 u rel-L2 <= 1e-4 and the force within 1e-4 of the oracle's (relative
to its magnitude); FP16 storage u <= 5e-3.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import rel_l2

pytestmark = pytest.mark.gpu


class Cyl:
    """Schafer-Turek channel with n_d cells per diameter, Re = 100."""

    def __init__(self, n_d=10, u_mean=0.05, re=100.0, bouzidi=True, inlet="zou_he"):
        self.lat = O.Lattice(9)
        m, self.center, self.radius, uin = I.schafer_turek_2d(n_d, u_mean)
        self.mask = m
        self.uin = uin.astype(np.float32)
        self.omega = 1.0 / (3.0 * u_mean * n_d / re + 0.5)
        cells, dirs, q = I.ball_links(m, self.center, self.radius, self.lat.c)
        self.cells, self.dirs, self.q = cells, dirs, q.astype(np.float32)
        self.bouzidi = bouzidi
        self.inlet = inlet
        wq = np.full((9,) + m.shape, np.nan)
        if bouzidi:
            yy, xx = np.unravel_index(cells, m.shape)
            wq[dirs, yy, xx] = self.q.astype(np.float64)
        self.rho0 = np.ones(m.shape)
        self.u0 = self.uin.astype(np.float64) * O.fluid_like(m)
        self.p = O.Params(self.lat, self.omega,
                          bc=O.BC(2, inlet_u=self.uin.astype(np.float64), wall_q=wq if bouzidi else None,
                                  inlet_scheme=inlet))
        yy, xx = np.meshgrid(np.arange(m.shape[0]), np.arange(m.shape[1]), indexing="ij")
        self.body = ((xx - self.center[0]) ** 2 + (yy - self.center[1]) ** 2 <= self.radius ** 2) & (m == O.WALL)

    def gpu(self, storage="f32"):
        ny, nx = self.mask.shape
        s = X.Simulation(9, (nx, ny), self.omega, "bgk", storage)
        s.set_mask(self.mask)
        s.set_inlet_profile(self.uin)
        s.set_inlet_scheme(self.inlet)
        if self.bouzidi:
            s.set_wall_distances(self.cells, self.dirs, self.q)
        s.init(self.rho0.astype(np.float32), self.u0.astype(np.float32))
        return s


@pytest.mark.parametrize("bouzidi,inlet", [(True, "zou_he"), (False, "zou_he"), (True, "regularized")])
def test_cylinder_parity_fp32(bouzidi, inlet):
    c = Cyl(bouzidi=bouzidi, inlet=inlet)
    s = c.gpu()
    f = O.init_state(c.lat, c.rho0, c.u0, c.mask, c.p)
    for _ in range(4):
        # the GPU reports the force of its latest update (step t-1 -> t);
        # the oracle's force is that of the update starting from f_{t-1}
        s.step(100)
        f = O.run(c.lat, f, c.mask, c.p, 99)
        Fo = O.wall_force(c.lat, f, c.mask, c.p, solid=c.body)
        f = O.step(c.lat, f, c.mask, c.p)
        Fg = s.wall_force()
        assert np.max(np.abs(Fg[:2] - Fo)) <= 1e-4 * np.max(np.abs(Fo)), (Fg, Fo)
        assert Fg[2] == 0.0
    _, ug = s.macroscopic()
    _, uo = O.macroscopic(c.lat, f, c.mask, c.p)
    fl = O.fluid_like(c.mask)
    assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-4
    s.close()


def test_cylinder_parity_fp16():
    c = Cyl()
    s = c.gpu("f16")
    s.step(400)
    _, ug = s.macroscopic()
    s.close()
    f = O.run(c.lat, O.init_state(c.lat, c.rho0, c.u0, c.mask, c.p), c.mask, c.p, 400)
    _, uo = O.macroscopic(c.lat, f, c.mask, c.p)
    fl = O.fluid_like(c.mask)
    assert rel_l2(ug[:, fl], uo[:, fl]) <= 5e-3


@pytest.mark.parametrize("q,coll,inlet", [(19, "bgk", "zou_he"), (19, "bgk", "regularized"),
                                          (27, "kbc", "regularized")])
def test_sphere_bouzidi_3d(q, coll, inlet):
    """A sphere of radius 3.27 between an INLET and an OUTLET plane, periodic
    in y and z, constant inflow, Bouzidi links on the sphere."""
    lat = O.Lattice(q)
    nx, ny, nz = 40, 16, 14
    center, radius = (12.3, 7.6, 6.8), 3.27
    m = np.zeros((nz, ny, nx), np.uint8)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ball = (xx - center[0]) ** 2 + (yy - center[1]) ** 2 + (zz - center[2]) ** 2 <= radius ** 2
    m[ball] = O.WALL
    m[:, :, 0] = O.INLET
    m[:, :, -1] = O.OUTLET
    cells, dirs, qd = I.ball_links(m, center, radius, lat.c)
    qd = qd.astype(np.float32)
    wq = np.full((lat.q,) + m.shape, np.nan)
    wq[(dirs,) + np.unravel_index(cells, m.shape)] = qd
    uin = (0.04, 0.0, 0.0)
    p = O.Params(lat, 1.6, collision=coll, bc=O.BC(3, inlet_u=uin, wall_q=wq, inlet_scheme=inlet))
    u0 = np.zeros((3,) + m.shape)
    u0[0][O.fluid_like(m)] = uin[0]
    f = O.run(lat, O.init_state(lat, np.ones(m.shape), u0, m, p), m, p, 149)
    Fo = O.wall_force(lat, f, m, p)          # the update 149 -> 150
    f = O.step(lat, f, m, p)
    _, uo = O.macroscopic(lat, f, m, p)
    s = X.Simulation(q, (nx, ny, nz), 1.6, coll, "f32")
    s.set_mask(m)
    s.set_bc(X.XLB_CELL_INLET, 1.0, uin)
    s.set_inlet_scheme(inlet)
    s.set_wall_distances(cells, dirs, qd)
    s.init(np.ones(m.shape, np.float32), u0.astype(np.float32))
    s.step(150)
    _, ug = s.macroscopic()
    Fg = s.wall_force()
    s.close()
    fl = O.fluid_like(m)
    assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-4
    assert np.max(np.abs(Fg - Fo)) <= 1e-4 * np.max(np.abs(Fo))


def test_wall_force_to_device_and_argument_checks():
    torch = pytest.importorskip("torch")
    c = Cyl()
    s = c.gpu()
    with pytest.raises(X.XlbError):
        s.wall_force()                               # no post-collision state yet
    s.step(20)
    host = s.wall_force()
    dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    s.wall_force(dev)
    s.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)
    fluid = int(np.flatnonzero(c.mask.ravel() == O.FLUID)[0])
    with pytest.raises(X.XlbError):
        s.set_wall_distances([fluid], [1], [0.5])    # not a link to a WALL cell
    with pytest.raises(X.XlbError):
        s.set_wall_distances(c.cells[:1], c.dirs[:1], [1.5])   # q out of range
    s.set_wall_distances([], [], [])                 # clears the list
    s.close()
    s = X.Simulation(9, (16, 16), 1.2, "bgk", "f32")
    with pytest.raises(X.XlbError):
        s.set_wall_distances([0], [1], [0.5])        # no mask yet
    s.close()


def schafer_turek_coefficients(n_d=80, u_mean=0.003, t_end=100.0, every=100, storage="f32"):
    """The Section 4.3 run: Schafer-Turek 2D cylinder, Re = 100, n_d cells per
    diameter, mean inflow u_mean (lattice units), BGK, Bouzidi cylinder,
    regularized Poiseuille inflow, outflow, halfway walls; t in units of D/U.
    (With the Zou-He inflow rule this run diverges near the inlet after about
    5,000 steps at 80 cells per diameter, in the oracle's arithmetic as on the
    GPU; Section 4.3 allows either rule.)  Returns (t, C_d(t), C_l(t)) sampled
    every `every` steps, the force series written on the device without host
    round trips."""
    import torch
    c = Cyl(n_d=n_d, u_mean=u_mean, inlet="regularized")
    s = c.gpu(storage)
    s.set_step_graph(every)
    steps = int(round(t_end * n_d / u_mean))
    n = steps // every
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    s.step(1)
    base = F.data_ptr()
    for k in range(n):
        s.step(every)
        s.wall_force(base + 24 * k)
    s.synchronize()
    s.close()
    Fh = F.cpu().numpy()
    t = (1 + every * (np.arange(n) + 1)) * u_mean / n_d
    scale = 2.0 / (u_mean * u_mean * n_d)          # 2 F / (rho U^2 D), rho = 1
    return t, scale * Fh[:, 0], scale * Fh[:, 1]


def strouhal(t, cl):
    """Shedding frequency D f / U from the mean period between upward zero
    crossings of C_l (linear interpolation)."""
    x = cl - cl.mean()
    k = np.flatnonzero((x[:-1] < 0) & (x[1:] >= 0))
    tc = t[k] - x[k] * (t[k + 1] - t[k]) / (x[k + 1] - x[k])
    return (len(tc) - 1) / (tc[-1] - tc[0])


def test_schafer_turek_paper_coefficients():
    """Section 4.3 prints C_d^max = 3.25, C_l^max = 0.985 (over t <= 100) and
    St = 0.300 (from C_l on 50 <= t <= 100) at 80 cells per diameter,
    u_LB = 0.003; the benchmark's reference ranges are 3.22-3.24, 0.99-1.01
    and 0.295-0.305.  Maxima here are taken over the periodic window
    50 <= t <= 100."""
    pytest.importorskip("torch")
    t, cd, cl = schafer_turek_coefficients()
    win = t >= 50.0
    cd_max, cl_max, st = cd[win].max(), cl[win].max(), strouhal(t[win], cl[win])
    print(f"Schafer-Turek 2D-2, 80 cells/D: Cd_max={cd_max:.4f} Cl_max={cl_max:.4f} St={st:.4f}")
    assert abs(cd_max - 3.25) <= 0.05
    assert abs(cl_max - 0.985) <= 0.05
    assert abs(st - 0.300) <= 0.009
