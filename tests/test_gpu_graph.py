"""Graph replay of the update (xlb_set_step_graph) gives the same populations,
bit for bit, as launching every update, including after boundary changes
(which force a new capture) and with an odd number of updates per graph
(both starting buffers get a graph)."""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import Case

pytestmark = pytest.mark.gpu


def _mixed_case():
    sh = (40, 72)
    m = I.channel_2d_mask(72, 40, top=O.LID)
    m[I.random_obstacle_mask(sh, 0.05, seed=51) > 0] = O.WALL
    m[I.random_obstacle_mask(sh, 0.03, seed=52) > 0] = O.FWALL
    m[I.random_obstacle_mask(sh, 0.02, seed=53) > 0] = O.EQ
    m[0, :] = O.WALL
    m[-1, :] = O.LID
    r, u = I.random_flow(sh, 2, seed=54, rho_amp=0.005, u_amp=0.02)
    return Case(9, sh, 1.5, "bgk", mask=m, force=(1e-5, 0.0, 0.0), lid=(1.0, (0.04, 0.0, 0.0)),
                eq=(1.0, (0.01, 0.0, 0.0)), rho0=r, u0=u)


@pytest.mark.parametrize("g", [1, 7, 20])
def test_graph_replay_is_bit_identical(g):
    c = _mixed_case()
    a = c.gpu_sim()
    b = c.gpu_sim()
    b.set_step_graph(g)
    for sim in (a, b):
        sim.step(101)
    pa, ka = a.populations()
    pb, kb = b.populations()
    assert ka == kb == 1 and np.array_equal(pa, pb)
    assert a.time == b.time == 101
    # new boundary values: the graph is captured again
    for sim in (a, b):
        sim.set_bc(X.XLB_CELL_LID, 1.0, (-0.03, 0.01, 0.0))
        sim.step(45)
    pa, _ = a.populations()
    pb, _ = b.populations()
    assert np.array_equal(pa, pb)
    a.close()
    b.close()


def test_graph_replay_taylor_green_3d():
    """Periodic D3Q19 (bulk kernel only), 16-bit storage, g = 50."""
    sh = (16, 24, 32)
    r, u = I.random_flow(sh, 3, seed=55, rho_amp=0.01, u_amp=0.03)
    c = Case(19, sh, 1.3, "bgk", rho0=r, u0=u)
    a = c.gpu_sim("f16")
    b = c.gpu_sim("f16")
    b.set_step_graph(50)
    a.step(300)
    b.step(300)
    assert np.array_equal(a.populations()[0], b.populations()[0])
    a.close()
    b.close()


def test_graph_argument_check():
    c = _mixed_case()
    s = c.gpu_sim()
    with pytest.raises(X.XlbError):
        s.set_step_graph(-1)
    s.set_step_graph(0)
    s.step(3)
    s.close()


def test_graph_replay_with_curved_walls_and_inflow():
    """The Section 4.3 set-up (Bouzidi links, inflow profile, regularized
    inlet, outflow) steps identically with and without graph replay, and the
    wall force of the last update agrees bit for bit."""
    from test_gpu_cylinder import Cyl
    c = Cyl(n_d=10, u_mean=0.05, inlet="regularized")
    a = c.gpu()
    b = c.gpu()
    b.set_step_graph(9)
    for sim in (a, b):
        sim.step(95)
    assert np.array_equal(a.populations()[0], b.populations()[0])
    assert np.array_equal(a.wall_force(), b.wall_force())
    a.close()
    b.close()
