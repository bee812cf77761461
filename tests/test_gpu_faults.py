"""Failure detection on the host side of the library (no GPU fault is
provoked): allocation failure reported as XLB_ERR_OOM with the context still
usable, invalid arguments, and a non-finite state showing up in the FP64
reductions.  No kernel of the library waits on another block or on the
host, so there is no device-side timeout to run out."""
import math

import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X

pytestmark = pytest.mark.gpu


def test_tape_allocation_failure_is_oom_and_recoverable():
    s = X.Simulation(19, (32, 32, 32), 1.2, "bgk", "f32")
    s.init()
    with pytest.raises(X.XlbError) as ei:
        X.xlb_tape_begin(s.ctx, 1_000_000, 1)       # ~2.5 TB of checkpoints
    assert ei.value.status == X.XLB_ERR_OOM
    with pytest.raises(X.XlbError) as ei:
        X.xlb_tape_begin(s.ctx, 2 ** 62, 1)         # size overflow, refused before allocating
    assert ei.value.status == X.XLB_ERR_OOM
    # the context still works: a small tape, steps, a reduction
    X.xlb_tape_begin(s.ctx, 4, 2)
    s.step(4)
    X.xlb_tape_end(s.ctx)
    mass, _ = s.reduce()
    assert abs(mass - 32 ** 3) < 1e-6 * 32 ** 3
    s.close()


def test_invalid_arguments_leave_state_unchanged():
    m = I.lid_driven_cavity_mask(12)
    s = X.Simulation(19, (12, 12, 12), 1.2, "bgk", "f32")
    s.set_mask(m)
    s.init()
    s.step(3)
    before = s.populations()[0].copy()
    bad = m.copy()
    bad[5, 5, 5] = 9
    with pytest.raises(X.XlbError) as ei:
        s.set_mask(bad)
    assert ei.value.status == X.XLB_ERR_ARG
    with pytest.raises(X.XlbError):
        s.step(-1)
    with pytest.raises(X.XlbError):
        X.xlb_set_bc(s.ctx, X.XLB_CELL_WALL, 1.0, (0.0, 0.0, 0.0))
    assert np.array_equal(s.populations()[0], before)
    s.close()
    with pytest.raises(X.XlbError):
        X.Simulation(19, (0, 4, 4), 1.2, "bgk", "f32")
    with pytest.raises(X.XlbError):
        X.Simulation(19, (8, 8, 8), 1.2, "kbc", "f32")   # KBC needs D2Q9 / D3Q27


def test_non_finite_state_shows_in_reductions():
    """A NaN written into one population (host-side injection through the
    state API) spreads with the flow and is reported by the FP64 mass sum."""
    s = X.Simulation(9, (32, 24), 1.3, "bgk", "f32")
    s.init()
    s.step(2)
    buf = s.state_get().copy()
    data = buf[64:].view(np.float32)
    data[100] = np.nan
    s.state_set(buf)
    s.step(5)
    mass, mom = s.reduce()
    assert math.isnan(mass)
    rho, _ = s.macroscopic()
    assert np.isnan(rho).any() and np.isfinite(rho).any()
    s.close()
