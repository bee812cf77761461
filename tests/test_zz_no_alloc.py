"""The allocation-free moments entry point, through the C ABI.

xlb_moments_noalloc serves callers that cannot call cudaMalloc (latency-
critical loops, where the allocator may synchronise the device; host
frameworks that own all device memory through their own pools; recovery
paths after the device ran out of memory): its partial sums live in a fixed
array inside the library.  Each check calls it twice in a row on the same
populations and compares the result with two references:

* a host FP64 sum of the stored populations, read back with xlb_state_get
  and weighted with the oracle's lattice tables (independent of the library);
* xlb_reduce, where both sum the same state (right after initialisation, and
  after steps on a periodic lattice, where the post-collision totals equal
  the post-stream ones).

On a walled cavity after several steps the live buffer holds post-collision
populations, whose momentum differs from xlb_reduce's post-stream totals;
that case is compared with the host sum only.  The tolerance is FP64
summation order, 1e-12 relative.  This file is collected last, so that a run
stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X

pytestmark = pytest.mark.gpu


def _host_totals(sim, mask):
    """FP64 (mass, j_x, j_y, j_z) of the stored populations over fluid-like
    cells, summed on the host from a state snapshot."""
    raw, _ = sim.populations()
    if sim.storage == X.XLB_STORE_BF16:
        df = (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        df = raw.astype(np.float64)
    lat = O.Lattice(sim.Q)
    f = df + lat.w.reshape((-1,) + (1,) * (df.ndim - 1))
    sel = np.ones(df.shape[1:], bool) if mask is None else np.isin(mask, O.FLUID_LIKE)
    out = [float(f.sum(axis=0)[sel].sum())]
    for a in range(3):
        ca = lat.c[:, a] if a < lat.d else np.zeros(lat.q)
        out.append(float(np.tensordot(ca.astype(float), f, axes=(0, 0))[sel].sum()))
    return np.array(out)


def _call_twice(sim, mask_dev, out, stream=None):
    # the simulation works on its own stream: let it finish before another
    # stream reads its populations
    sim.synchronize()
    ptr, plane = X.xlb_populations(sim.ctx)
    res = []
    for _ in range(2):  # two calls in a row share the fixed scratch
        if isinstance(out, torch.Tensor):
            out.fill_(np.nan)
        else:
            out[:] = np.nan
        X.xlb_moments_noalloc(sim.Q, sim.dims, sim.storage, ptr, plane, mask_dev, out,
                              None if stream is None else stream.cuda_stream)
        if isinstance(out, torch.Tensor):
            torch.cuda.synchronize()
            res.append(out.cpu().numpy().copy())
        else:
            res.append(out.copy())
    return res


def _assert_close(got, ref):
    scale = abs(ref[0])
    for k in range(4):
        assert abs(got[k] - ref[k]) <= 1e-12 * scale, (k, got, ref)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_noalloc_matches_host_sum_and_reduce_periodic(storage):
    shape = (12, 20, 40)
    rho, u = I.random_flow(shape, 3, seed=11, rho_amp=0.01, u_amp=0.03)
    sim = X.Simulation(19, tuple(reversed(shape)), 1.6, "bgk", storage)
    sim.init(rho.astype(np.float32), u.astype(np.float32))
    for got in _call_twice(sim, None, np.zeros(4)):  # pre-collision state, host out
        _assert_close(got, _host_totals(sim, None))
        mass, mom = sim.reduce()
        _assert_close(got, np.array([mass] + list(mom)))
    sim.step(15)  # post-collision state: on a periodic lattice its totals are f_t's
    for got in _call_twice(sim, None, torch.zeros(4, dtype=torch.float64, device="cuda")):
        _assert_close(got, _host_totals(sim, None))
        mass, mom = sim.reduce()
        _assert_close(got, np.array([mass] + list(mom)))
    sim.close()


def test_noalloc_sums_the_stored_state_of_a_walled_cavity():
    """Fluid-like cells only, on a lid-driven cavity: right after
    initialisation (where the stored state is the post-stream state that
    xlb_reduce sums) and after 7 steps (where it is the post-collision
    state, compared with the host sum of the same populations)."""
    m = I.lid_driven_cavity_mask(24, 18, 16)
    rho, u = I.random_flow(m.shape, 3, seed=12, rho_amp=0.01, u_amp=0.02)
    sim = X.Simulation(19, tuple(reversed(m.shape)), 1.5, "bgk", "f32")
    sim.set_mask(m)
    sim.set_bc(X.XLB_CELL_LID, 1.0, (0.05, 0.0, 0.0))
    sim.init(rho.astype(np.float32), u.astype(np.float32))
    mdev = torch.from_numpy(m.reshape(-1)).cuda()
    for got in _call_twice(sim, mdev, np.zeros(4)):
        _assert_close(got, _host_totals(sim, m))
        mass, mom = sim.reduce()
        _assert_close(got, np.array([mass] + list(mom)))
    sim.step(7)
    ref = _host_totals(sim, m)
    for got in _call_twice(sim, mdev, torch.zeros(4, dtype=torch.float64, device="cuda")):
        _assert_close(got, ref)
    sim.close()


def test_noalloc_runs_on_the_callers_stream():
    """A caller's own (non-default) stream: the simulation runs on it and
    the entry point queues its kernels on it, with the result in device
    memory."""
    shape = (16, 16, 32)
    rho, u = I.random_flow(shape, 3, seed=13, rho_amp=0.01, u_amp=0.03)
    s = torch.cuda.Stream()
    sim = X.Simulation(19, tuple(reversed(shape)), 1.4, "bgk", "f32", stream=s.cuda_stream)
    sim.init(rho.astype(np.float32), u.astype(np.float32))
    sim.step(3)
    torch.cuda.synchronize()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for got in _call_twice(sim, None, out, stream=s):
        _assert_close(got, _host_totals(sim, None))
    sim.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    pop = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = np.zeros(4)
    with pytest.raises(X.XlbError) as e:  # 512 x 512 x 512 cells > 67,108,864
        X.xlb_moments_noalloc(19, (512, 512, 512), X.XLB_STORE_F32, pop, 512 ** 3, None, out)
    assert e.value.status == X.XLB_ERR_ARG
    with pytest.raises(X.XlbError) as e:  # a product of extents that overflows 64 bits
        X.xlb_moments_noalloc(19, (1 << 26, 1 << 26, 1 << 26), X.XLB_STORE_F32, pop, 1 << 62, None, out)
    assert e.value.status == X.XLB_ERR_ARG
    with pytest.raises(X.XlbError):
        X.xlb_moments_noalloc(19, (4, 4, 4), X.XLB_STORE_F32, pop, 10, None, out)  # stride < N
