"""GPU adjoint (reverse mode through the C ABI) against the FP64 oracle's
hand-derived adjoint and against the oracle's central finite differences.

Bars: GPU gradient vs oracle adjoint, relative L2 <= 1e-4; GPU directional
derivative vs oracle central FD, relative <= 1e-3 per direction.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import Case, rel_l2

pytestmark = pytest.mark.gpu


def _case(q, shape, walls, force, seed=21):
    lat = O.Lattice(q)
    d = lat.d
    if walls:
        mask = I.lid_driven_cavity_mask(shape[-1], shape[-2], shape[0]) if d == 3 else \
            I.channel_2d_mask(shape[1], shape[0], top=O.LID)
    else:
        mask = np.zeros(shape, np.uint8)
    rho0 = 1.0 + I.density_perturbation(shape, 1e-3, seed=seed)
    u0 = I.random_flow(shape, d, seed=seed + 1, u_amp=0.02)[1]
    return Case(q, shape, 1.4, "bgk", mask=mask, force=force,
                lid=(1.0, (0.05, 0.0, 0.0)) if walls else None,
                rho0=rho0.astype(np.float32).astype(np.float64),
                u0=u0.astype(np.float32).astype(np.float64))


def _box(shape):
    return tuple(slice(n // 4, n - n // 4) for n in shape)


def gpu_gradient(c, steps, k, storage="f32"):
    sim = c.gpu_sim(storage)
    X.xlb_tape_begin(sim.ctx, steps, k)
    sim.step(steps)
    rho, u = sim.macroscopic()
    rb, ub = O.kinetic_energy_grads(rho.astype(np.float64), u.astype(np.float64), _box(c.shape))
    X.xlb_adjoint_seed_macro(sim.ctx, rb.astype(np.float32), ub.astype(np.float32))
    X.xlb_adjoint_step(sim.ctx, steps)
    g_rho = np.empty(c.shape, np.float32)
    g_u = np.empty((c.lat.d,) + c.shape, np.float32)
    X.xlb_adjoint_init_grad(sim.ctx, g_rho, g_u)
    X.xlb_tape_end(sim.ctx)
    sim.close()
    return g_rho.astype(np.float64), g_u.astype(np.float64)


def oracle_gradient(c, steps):
    p = c.params()
    box = _box(c.shape)
    return O.gradient_init(c.lat, c.rho0, c.u0, c.mask, p, steps,
                           lambda r, u: O.kinetic_energy_grads(r, u, box))


def oracle_loss(c, rho0, steps):
    p = c.params()
    f = O.run(c.lat, O.init_state(c.lat, rho0, c.u0, c.mask, p), c.mask, p, steps)
    return O.kinetic_energy(c.lat, f, c.mask, p, _box(c.shape))


@pytest.mark.parametrize("q,shape,steps,walls,force", [
    (9, (40, 48), 60, False, None),
    (9, (34, 40), 60, True, (1e-5, 0.0, 0.0)),
    (19, (16, 16, 24), 40, False, None),
    (19, (18, 18, 18), 40, True, None),
])
def test_adjoint_matches_oracle_adjoint(q, shape, steps, walls, force):
    c = _case(q, shape, walls, force)
    g_rho, g_u = gpu_gradient(c, steps, k=7)
    o_rho, o_u = oracle_gradient(c, steps)
    fl = O.fluid_like(c.mask)
    assert rel_l2(g_rho[fl], o_rho[fl]) <= 1e-4
    assert rel_l2(g_u[:, fl], o_u[:, fl]) <= 1e-4


def test_checkpoint_interval_does_not_change_gradient():
    c = _case(19, (12, 12, 16), True, None)
    a, _ = gpu_gradient(c, 30, k=1)
    b, _ = gpu_gradient(c, 30, k=7)
    d, _ = gpu_gradient(c, 30, k=30)
    assert np.array_equal(a, b) and np.array_equal(a, d)


def test_adjoint_matches_central_differences():
    """The gradient of the kinetic energy in the central box with respect to
    the initial density, dotted with random directions, against FP64 central
    differences of the oracle (eps = 1e-6), 16 directions."""
    c = _case(19, (16, 16, 16), False, None, seed=5)
    steps = 40
    g_rho, _ = gpu_gradient(c, steps, k=10)
    rng = np.random.default_rng(77)
    eps = 1e-6
    for _ in range(16):
        d = rng.standard_normal(c.shape)
        fd = (oracle_loss(c, c.rho0 + eps * d, steps) - oracle_loss(c, c.rho0 - eps * d, steps)) / (2 * eps)
        assert abs(float((g_rho * d).sum()) - fd) <= 1e-3 * abs(fd)


def test_repeated_gradients_reuse_the_tape():
    """Two gradients in a row on one context (the second reuses the tape
    memory kept after xlb_tape_end) are identical; a larger tape afterwards
    grows the memory and still matches a fresh context."""
    c = _case(9, (24, 32), True, None)
    sim = c.gpu_sim()
    box = _box(c.shape)

    def grad(steps, k):
        sim.init(np.ascontiguousarray(c.rho0, dtype=np.float32), np.ascontiguousarray(c.u0, dtype=np.float32))
        X.xlb_tape_begin(sim.ctx, steps, k)
        sim.step(steps)
        rho, u = sim.macroscopic()
        rb, ub = O.kinetic_energy_grads(rho.astype(np.float64), u.astype(np.float64), box)
        X.xlb_adjoint_seed_macro(sim.ctx, rb.astype(np.float32), ub.astype(np.float32))
        X.xlb_adjoint_step(sim.ctx, steps)
        g = np.empty(c.shape, np.float32)
        X.xlb_adjoint_init_grad(sim.ctx, g, None)
        X.xlb_tape_end(sim.ctx)
        return g

    a = grad(30, 5)
    b = grad(30, 5)
    assert np.array_equal(a, b)
    big = grad(50, 10)
    X.xlb_tape_release(sim.ctx)
    sim.close()
    fresh, _ = gpu_gradient(c, 50, 10)
    assert np.array_equal(big, fresh)


def test_adjoint_state_errors():
    c = _case(9, (16, 16), False, None)
    sim = c.gpu_sim()
    with pytest.raises(X.XlbError):
        X.xlb_adjoint_step(sim.ctx, 1)          # no tape
    X.xlb_tape_begin(sim.ctx, 5, 2)
    sim.step(3)
    with pytest.raises(X.XlbError):
        X.xlb_adjoint_seed_macro(sim.ctx, None, None)  # not all taped steps taken
    with pytest.raises(X.XlbError):
        sim.step(3)                              # past the tape
    sim.close()
