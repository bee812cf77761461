"""The allocation-free moments entry point against xlb_reduce.

xlb_moments_noalloc serves callers that must not allocate device memory
(graph capture, pre-allocated real-time loops, hosts with their own memory
pools): its partial sums live in a fixed array inside the library.  Here it
is called through the C ABI twice in a row on the same populations and must
agree with xlb_reduce (which uses per-context scratch) to FP64 summation
order, 1e-12 relative.  This file is collected last so that a run stopping at
its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X

pytestmark = pytest.mark.gpu


def _close(a, b, scale):
    return abs(a - b) <= 1e-12 * scale


def _check(sim, mask_dev, storage, out):
    ptr, plane = X.xlb_populations(sim.ctx)
    mass, mom = sim.reduce()
    for _ in range(2):  # two calls in a row share the fixed scratch
        if isinstance(out, torch.Tensor):
            out.zero_()
        else:
            out[:] = 0.0
        X.xlb_moments_noalloc(sim.Q, sim.dims, X.STORAGE[storage], ptr, plane, mask_dev, out)
        if isinstance(out, torch.Tensor):
            torch.cuda.synchronize()
            got = out.cpu().numpy()
        else:
            got = out
        assert _close(got[0], mass, mass)
        for a in range(3):
            assert _close(got[1 + a], mom[a], mass)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_noalloc_matches_reduce_periodic(storage):
    shape = (12, 20, 40)
    rho, u = I.random_flow(shape, 3, seed=11, rho_amp=0.01, u_amp=0.03)
    sim = X.Simulation(19, tuple(reversed(shape)), 1.6, "bgk", storage)
    sim.init(rho.astype(np.float32), u.astype(np.float32))
    _check(sim, None, storage, np.zeros(4))                        # pre-collision state, host out
    sim.step(15)                                                   # post-collision state: periodic
    _check(sim, None, storage, torch.zeros(4, dtype=torch.float64, device="cuda"))  # device out
    sim.close()


def test_noalloc_matches_reduce_with_mask():
    """Fluid-like cells only, on a cavity right after initialisation (the
    stored populations are the post-stream state the reduction sums)."""
    m = I.lid_driven_cavity_mask(24, 18, 16)
    rho, u = I.random_flow(m.shape, 3, seed=12, rho_amp=0.01, u_amp=0.02)
    sim = X.Simulation(19, tuple(reversed(m.shape)), 1.5, "bgk", "f32")
    sim.set_mask(m)
    sim.init(rho.astype(np.float32), u.astype(np.float32))
    mdev = torch.from_numpy(m.reshape(-1)).cuda()
    _check(sim, mdev, "f32", np.zeros(4))
    sim.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    pop = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = np.zeros(4)
    with pytest.raises(X.XlbError) as e:  # 512 x 512 x 512 cells > 67,108,864
        X.xlb_moments_noalloc(19, (512, 512, 512), X.XLB_STORE_F32, pop, 512 ** 3, None, out)
    assert e.value.status == X.XLB_ERR_ARG
    with pytest.raises(X.XlbError):
        X.xlb_moments_noalloc(19, (4, 4, 4), X.XLB_STORE_F32, pop, 10, None, out)  # stride < N
