"""BF16 storage rounds stochastically; FP16 rounds to nearest even.

One BGK update from a state that BF16 represents exactly is taken twice:
with FP32 storage (which keeps the FP32 post-collision values the kernel
computes) and with BF16 storage.  Both run the same FP32 arithmetic on the
same inputs, so every BF16 result must be one of the two BF16 neighbours of
the FP32 value, rounded up with probability equal to the discarded fraction
(unbiased), and the same on every run.  FP16 results must be the FP32 values
rounded to nearest even.
"""
import numpy as np
import pytest

from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X

pytestmark = pytest.mark.gpu

SHAPE = (16, 20, 24)


def _state(sim, raw, kind_h=1):
    buf = sim.state_get().copy()
    buf[:64].view(np.int32)[12] = kind_h
    data = buf[64:].view(raw.dtype)
    align = 256 // raw.itemsize
    plane = (sim.N + align - 1) // align * align
    data.reshape(sim.Q, plane)[:, :sim.N] = raw.reshape(sim.Q, sim.N)
    sim.state_set(buf)


def _one_step(storage, raw):
    sim = X.Simulation(19, tuple(reversed(SHAPE)), 1.3, "bgk", storage)
    sim.init()
    _state(sim, raw)
    sim.step(1)
    got, kind = sim.populations()
    assert kind == 1
    sim.close()
    return got.copy()


def _bf16_exact_state():
    rho, u = I.random_flow(SHAPE, 3, seed=5, rho_amp=0.02, u_amp=0.05)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    c = np.array(X.xlb_lattice_table(19)[0])
    usq = (u ** 2).sum(0)
    df = np.stack([w[i] * ((rho - 1) + rho * (3 * np.tensordot(c[i], u, 1) + 4.5 * np.tensordot(c[i], u, 1) ** 2
                                               - 1.5 * usq)) for i in range(19)])
    df *= 1.0 + 0.1 * np.random.default_rng(6).uniform(-1, 1, df.shape)  # off equilibrium
    b16 = (df.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)  # exact in BF16
    f32 = (b16.astype(np.uint32) << 16).view(np.float32)
    return b16, f32


def test_bf16_rounding_is_stochastic_and_unbiased():
    b16, f32 = _bf16_exact_state()
    ref = _one_step("f32", f32).view(np.uint32)          # exact FP32 post-collision values
    got = _one_step("bf16", b16).astype(np.uint32)
    again = _one_step("bf16", b16).astype(np.uint32)
    assert np.array_equal(got, again)                    # reproducible
    lo = ref >> 16                                       # truncated magnitude
    frac = (ref & 0xFFFF) / 65536.0
    up = got == lo + 1
    assert np.all((got == lo) | up)                      # one of the two neighbours
    assert not np.any(up & (frac == 0.0))                # exact values stay exact
    n = frac.size
    assert abs(up.mean() - frac.mean()) < 4.0 * 0.5 / np.sqrt(n)   # unbiased
    for a, b in ((0.0, 0.25), (0.25, 0.5), (0.5, 0.75), (0.75, 1.0)):
        sel = (frac > a) & (frac <= b)
        k = sel.sum()
        assert k > 1000
        assert abs(up[sel].mean() - frac[sel].mean()) < 4.0 * 0.5 / np.sqrt(k)


def test_f16_rounds_to_nearest_even():
    b16, f32 = _bf16_exact_state()
    h16 = f32.astype(np.float16)
    ref = _one_step("f32", h16.astype(np.float32))
    got = _one_step("f16", h16)
    assert np.array_equal(got.view(np.uint16), ref.astype(np.float16).view(np.uint16))
