"""Parity at the workloads' full sizes, in the launch configuration bench.py
times: sampled outputs the oracle computes one by one, and properties that
hold at any size.

- D3Q27 KBC sphere channel 512 x 256 x 256 (Zou-He inlet, outflow): one
  more update checked cell by cell on sampled cells (interior, sphere surface,
  inlet and outlet planes) against the oracle's C(S_bc(.)) on each cell's
  neighbourhood.
- D3Q19 adjoint, 128^3 periodic, 500 steps, checkpoints every 50: the
  gradient of the total mass with respect to the initial density is exactly 1
  and that of the total x-momentum with respect to u0_x is rho0 (mass and
  momentum are invariants of periodic BGK).
- 4096 batched channels: sampled domains against the oracle.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import Case, rel_l2

pytestmark = pytest.mark.gpu


def test_kbc_sphere_full_size_sampled_step():
    nx, ny, nz = 512, 256, 256
    mask = I.sphere_channel_mask(nx, ny, nz, radius=32, center=(128, 128, 128))
    uin = (0.04, 0.0, 0.0)
    u0 = np.zeros((3,) + mask.shape, np.float32)
    u0[0][O.fluid_like(mask)] = uin[0]
    c = Case(27, mask.shape, 1.857, "kbc", mask=mask, inlet=uin, rho0=np.ones(mask.shape, np.float32), u0=u0)
    sim = c.gpu_sim()
    sim.step(20)
    h_prev, _ = sim.populations()
    sim.step(1)
    h_next, _ = sim.populations()
    sim.close()
    rng = np.random.default_rng(1)
    pts = [tuple(int(v) for v in (rng.integers(0, nz), rng.integers(0, ny), rng.integers(2, nx - 2)))
           for _ in range(120)]
    pts += [(128, 128, 128 - 33), (128, 128 + 33, 128), (128 + 33, 128, 128), (100, 150, 110)]  # near the sphere
    pts += [(z, y, x) for (z, y) in ((0, 0), (5, 200), (255, 255)) for x in (0, 1, nx - 2, nx - 1)]
    lat, p = c.lat, c.params()
    w = lat.w[:, None, None, None]
    worst = 0.0
    for (z, y, x) in pts:
        if not O.fluid_like(mask[z, y, x]):
            continue
        zi = [(z + d) % nz for d in (-1, 0, 1)]
        yi = [(y + d) % ny for d in (-1, 0, 1)]
        xi = [(x + d) % nx for d in (-2, -1, 0, 1, 2)]  # the outflow reads the pull at x - 1
        idx = np.ix_(zi, yi, xi)
        hp = h_prev[(slice(None),) + idx].astype(np.float64) + w
        mp = mask[idx]
        f = O.stream_bc(lat, hp, mp, p.bc)
        hn = O.collide(lat, f, mp, p)[:, 1, 1, 2] - lat.w
        worst = max(worst, float(np.max(np.abs(h_next[:, z, y, x].astype(np.float64) - hn))))
    assert worst < 1e-6


def _gradients(seed_rho, seed_u, m=128, T=500, k=50):
    rho0 = (1.0 + I.density_perturbation((m, m, m), 1e-3, seed=1234)).astype(np.float32)
    u0 = I.random_flow((m, m, m), 3, seed=4, u_amp=0.01)[1].astype(np.float32)
    sim = X.Simulation(19, (m, m, m), 1.25, "bgk", "f32")
    sim.init(rho0, u0)
    X.xlb_tape_begin(sim.ctx, T, k)
    sim.step(T)
    rho, u = sim.macroscopic()
    X.xlb_adjoint_seed_macro(sim.ctx, seed_rho(rho, u), seed_u(rho, u))
    X.xlb_adjoint_step(sim.ctx, T)
    g_rho = np.empty((m, m, m), np.float32)
    g_u = np.empty((3, m, m, m), np.float32)
    X.xlb_adjoint_init_grad(sim.ctx, g_rho, g_u)
    X.xlb_tape_end(sim.ctx)
    sim.close()
    return rho0, u0, g_rho, g_u


def test_adjoint_full_size_mass_invariant():
    """L = sum rho_T: dL/drho0 = 1, dL/du0 = 0 everywhere."""
    _, _, g_rho, g_u = _gradients(lambda r, u: np.ones_like(r), lambda r, u: np.zeros_like(u))
    assert np.max(np.abs(g_rho - 1.0)) < 2e-5
    assert np.max(np.abs(g_u)) < 2e-5


def test_adjoint_full_size_momentum_invariant():
    """L = sum rho_T u_x,T = sum j_x: dL/drho0 = u0_x, dL/du0_x = rho0."""
    def sr(r, u):
        return u[0].copy()

    def su(r, u):
        s = np.zeros_like(u)
        s[0] = r
        return s

    rho0, u0, g_rho, g_u = _gradients(sr, su)
    assert np.max(np.abs(g_rho - u0[0])) < 2e-5
    assert np.max(np.abs(g_u[0] - rho0)) < 1e-4
    assert np.max(np.abs(g_u[1:])) < 2e-5


def test_batch_4096_sampled_domains():
    omega = 1.25
    doms = I.batched_channels(4096, seed=1234, nu=O.nu_from_omega(omega), u_max=0.05)
    b = X.Batch(doms, omega)
    b.set_masks()
    b.init()
    b.tune(10)
    b.step(200)
    got = b.macroscopic()
    b.close()
    cells = [d["nx"] * d["ny"] for d in doms]
    picks = {int(np.argmin(cells)), int(np.argmax(cells)), 1234, 4095}
    lat = O.Lattice(9)
    for k in picks:
        m = doms[k]["mask"]
        p = O.Params(lat, omega, force=doms[k]["force"])
        f = O.run(lat, O.init_state(lat, np.ones(m.shape), np.zeros((2,) + m.shape), m, p), m, p, 200)
        _, uo = O.macroscopic(lat, f, m, p)
        fl = m == 0
        assert rel_l2(got[k][1][:, fl], uo[:, fl]) <= 1e-4


def _crop_module():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_kbc_sphere_crop.py")
    spec = importlib.util.spec_from_file_location("make_kbc_sphere_crop", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("storage,tol", [("f32", 1e-4), ("f16", 5e-3), ("bf16", 5e-3)])
def test_kbc_sphere_crop_1000_steps_against_stored_oracle(storage, tol):
    """The KBC D3Q27 sphere channel scaled to 128 x 64 x 64 (radius 8), 1000
    steps, in the three storage forms, against the FP64 oracle's velocity
    stored by tests/golden/make_kbc_sphere_crop.py at 16,384 sampled fluid
    cells (relative L2 over the sample)."""
    mod = _crop_module()
    ref = np.load(mod.OUT)
    lat, mask, rho, u, p = mod.setup()
    assert np.array_equal(ref["index"], mod.sample_cells(mask))
    c = Case(27, mask.shape, mod.OMEGA, "kbc", mask=mask, inlet=(mod.U_IN, 0.0, 0.0), rho0=rho, u0=u)
    _, ug = c.gpu(int(ref["steps"]), storage)
    got = ug.reshape(3, -1)[:, ref["index"]].astype(np.float64)
    err = rel_l2(got, ref["u"])
    print(f"KBC crop {storage}: sampled rel-L2(u) after 1000 steps = {err:.3e}")
    assert err <= tol
