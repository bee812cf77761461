"""The differentiable rollout through torch.autograd, and the FP64 loss and
gradient-norm reductions on the GPU.

* xlb_kinetic_energy: against an FP64 host sum of the FP32 observables that
  xlb_macroscopic returns for the same state (1e-12: only the summation order
  differs) and against the oracle's loss (1e-4);
* xlb_sum_squares: against an FP64 host sum (1e-12);
* torch.autograd.grad through xlb.rollout (forward: tape + steps + loss;
  backward: the loss cotangent formed on the GPU, the adjoint, the gradient):
  against the oracle's hand-derived adjoint (relative L2 <= 1e-4) and against
  the oracle's central finite differences (relative <= 1e-3 per direction);
* the gradient workload's own tape structure (D3Q19 periodic, 500 steps,
  checkpoints every 50, central-box kinetic energy, Gaussian density
  perturbation of amplitude 1e-3), on a 24^3 lattice: the same two bars;
* the FP16 storage form of the adjoint against the oracle's adjoint at the
  storage bound (5e-3); BF16 storage is refused by the tape.
"""
import numpy as np
import pytest
import torch

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import Case, rel_l2

pytestmark = pytest.mark.gpu


def _oracle_loss(c, steps, box, rho0=None):
    p = c.params()
    f = O.init_state(c.lat, c.rho0 if rho0 is None else rho0, c.u0, c.mask, p)
    f = O.run(c.lat, f, c.mask, p, steps)
    return float(O.kinetic_energy(c.lat, f, c.mask, p, box))


@pytest.mark.parametrize("q", [9, 19])
def test_kinetic_energy_reduction(q):
    shape = (20, 28) if q == 9 else (10, 12, 16)
    d = 2 if q == 9 else 3
    mask = I.channel_2d_mask(shape[1], shape[0], top=O.LID) if q == 9 else \
        I.lid_driven_cavity_mask(shape[2], shape[1], shape[0])
    rho, u = I.random_flow(shape, d, seed=3, rho_amp=0.01, u_amp=0.03)
    c = Case(q, shape, 1.5, "bgk", mask=mask, lid=(1.0, (0.05, 0.0, 0.0)), force=(1e-5, 2e-6, 0.0),
             rho0=rho.astype(np.float32).astype(np.float64), u0=u.astype(np.float32).astype(np.float64))
    box = tuple(slice(1, n - 2) for n in shape)
    sim = c.gpu_sim()
    sim.step(25)
    loss = X.xlb_kinetic_energy(sim.ctx, box, sim.dims)
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    X.xlb_kinetic_energy(sim.ctx, box, sim.dims, dev)
    torch.cuda.synchronize()
    assert float(dev[0]) == loss
    r, uu = sim.macroscopic()
    host = 0.5 * (r.astype(np.float64) * (uu.astype(np.float64) ** 2).sum(0))[box].sum()
    assert abs(loss - host) <= 1e-12 * abs(host)
    ref = _oracle_loss(c, 25, box)
    assert abs(loss - ref) <= 1e-4 * abs(ref)
    sim.close()


def test_sum_squares():
    x = torch.randn(1_000_037, device="cuda", dtype=torch.float32)
    sim = X.Simulation(9, (8, 8), 1.0)
    got = X.xlb_sum_squares(sim.ctx, x)
    ref = float((x.double().cpu().numpy() ** 2).sum())
    assert abs(got - ref) <= 1e-12 * ref
    with pytest.raises(X.XlbError):
        X.xlb_sum_squares(sim.ctx, np.ones(4, np.float32))  # host memory
    sim.close()


def _grad_case(q, shape, walls, seed):
    d = 2 if q == 9 else 3
    if walls:
        mask = I.channel_2d_mask(shape[1], shape[0], top=O.LID) if d == 2 else \
            I.lid_driven_cavity_mask(shape[2], shape[1], shape[0])
    else:
        mask = np.zeros(shape, np.uint8)
    rho0 = (1.0 + I.density_perturbation(shape, 1e-3, seed=seed)).astype(np.float32).astype(np.float64)
    u0 = I.random_flow(shape, d, seed=seed + 1, u_amp=0.02)[1].astype(np.float32).astype(np.float64)
    return Case(q, shape, 1.4, "bgk", mask=mask, lid=(1.0, (0.05, 0.0, 0.0)) if walls else None,
                rho0=rho0, u0=u0)


def _autograd(c, steps, k, box, storage="f32", with_u=True):
    sim = c.gpu_sim(storage)
    rho0 = torch.tensor(c.rho0, dtype=torch.float32, device="cuda", requires_grad=True)
    u0 = torch.tensor(c.u0, dtype=torch.float32, device="cuda", requires_grad=True) if with_u else None
    loss = X.rollout(sim, rho0, steps, k, box, u0=u0)
    grads = torch.autograd.grad(loss, [rho0] + ([u0] if with_u else []))
    out = (float(loss.detach()),) + tuple(g.double().cpu().numpy() for g in grads)
    sim.close()
    return out


@pytest.mark.parametrize("q,shape,walls,steps,k", [(9, (24, 32), True, 40, 10), (19, (10, 12, 14), True, 30, 7),
                                                   (19, (12, 12, 12), False, 25, 25)])
def test_rollout_autograd_matches_oracle_adjoint_and_fd(q, shape, walls, steps, k):
    c = _grad_case(q, shape, walls, seed=31)
    box = tuple(slice(n // 4, n - n // 4) for n in shape)
    loss, g_rho, g_u = _autograd(c, steps, k, box)
    assert abs(loss - _oracle_loss(c, steps, box)) <= 1e-4 * abs(loss)
    p = c.params()
    go_rho, go_u = O.gradient_init(c.lat, c.rho0, c.u0, c.mask, p, steps,
                                   lambda r, u: O.kinetic_energy_grads(r, u, box))
    fl = O.fluid_like(c.mask)
    assert rel_l2(g_rho[fl], go_rho[fl]) <= 1e-4
    assert rel_l2(g_u[:, fl], go_u[:, fl]) <= 1e-4
    rng = np.random.default_rng(7)
    eps = 1e-6
    for _ in range(3):
        dirn = np.where(fl, rng.standard_normal(shape), 0.0)
        dirn /= np.linalg.norm(dirn)
        fd = (_oracle_loss(c, steps, box, c.rho0 + eps * dirn) - _oracle_loss(c, steps, box, c.rho0 - eps * dirn)) \
            / (2 * eps)
        assert abs((g_rho * dirn).sum() - fd) <= 1e-3 * abs(fd)


def test_gradient_workload_tape_structure():
    """D3Q19 periodic, omega 1.25, 500 steps with checkpoints every 50 (ten
    segments recomputed by the adjoint), kinetic energy of the central box
    (the middle quarter of each axis, as [48, 80) of 128), Gaussian density
    perturbation 1e-3 (seed 1234), u0 = 0: on a 24^3 lattice."""
    n = 24
    shape = (n, n, n)
    rho0 = (1.0 + I.density_perturbation(shape, 1e-3, seed=1234)).astype(np.float32).astype(np.float64)
    c = Case(19, shape, 1.25, "bgk", rho0=rho0)
    box = (slice(9, 15),) * 3
    loss, g_rho = _autograd(c, 500, 50, box, with_u=False)
    p = c.params()
    go_rho, _ = O.gradient_init(c.lat, c.rho0, c.u0, c.mask, p, 500,
                                lambda r, u: O.kinetic_energy_grads(r, u, box))
    assert rel_l2(g_rho, go_rho) <= 1e-4
    rng = np.random.default_rng(1234)
    eps = 1e-6
    for _ in range(4):
        dirn = rng.standard_normal(shape)
        dirn /= np.linalg.norm(dirn)
        fd = (_oracle_loss(c, 500, box, c.rho0 + eps * dirn) - _oracle_loss(c, 500, box, c.rho0 - eps * dirn)) \
            / (2 * eps)
        assert abs((g_rho * dirn).sum() - fd) <= 1e-3 * abs(fd)
    sim = X.Simulation(19, c.dims, 1.25)
    g = torch.tensor(g_rho, dtype=torch.float32, device="cuda")
    nrm2 = X.xlb_sum_squares(sim.ctx, g)
    assert abs(nrm2 - float((g.double() ** 2).sum())) <= 1e-12 * nrm2
    sim.close()


@pytest.mark.parametrize("q,shape", [(9, (24, 32)), (19, (10, 12, 14))])
def test_adjoint_with_fp16_storage(q, shape):
    """The adjoint of the FP16 forward (each rounding taken as the identity)
    against the FP64 oracle's adjoint, at the storage bound (5e-3)."""
    c = _grad_case(q, shape, walls=True, seed=41)
    box = tuple(slice(n // 4, n - n // 4) for n in shape)
    _, g_rho, g_u = _autograd(c, 30, 10, box, storage="f16")
    go_rho, go_u = O.gradient_init(c.lat, c.rho0, c.u0, c.mask, c.params(), 30,
                                   lambda r, u: O.kinetic_energy_grads(r, u, box))
    fl = O.fluid_like(c.mask)
    err = rel_l2(g_rho[fl], go_rho[fl])
    print(f"f16 adjoint rel-L2 = {err:.3e}")
    assert err <= 5e-3
    assert rel_l2(g_u[:, fl], go_u[:, fl]) <= 5e-3


def test_adjoint_refuses_bf16_storage():
    """With BF16 storage the gradient misses the storage bound (8e-3 on the
    D2Q9 case above), so the tape is refused."""
    sim = X.Simulation(9, (16, 12), 1.4, "bgk", "bf16")
    sim.init()
    with pytest.raises(X.XlbError) as e:
        X.xlb_tape_begin(sim.ctx, 10, 5)
    assert e.value.status == X.XLB_ERR_UNSUPPORTED
    sim.close()
