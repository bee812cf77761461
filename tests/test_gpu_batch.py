"""Batched small D2Q9 domains: the persistent launch against the FP64 oracle
domain by domain, against the one-launch-per-domain baseline (bit-exact),
across launch shapes, and the autotuner's contract (it leaves the state
unchanged)."""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import rel_l2

pytestmark = pytest.mark.gpu

OMEGA = 1.25


def _domains(n=8, seed=7):
    return I.batched_channels(n, seed=seed, nx_range=(16, 48), ny_range=(12, 34), radius=(2, 4),
                              nu=O.nu_from_omega(OMEGA), u_max=0.05)


def _oracle(dom, steps):
    lat = O.Lattice(9)
    m = dom["mask"]
    p = O.Params(lat, OMEGA, force=dom["force"])
    f = O.init_state(lat, np.ones(m.shape), np.zeros((2,) + m.shape), m, p)
    f = O.run(lat, f, m, p, steps)
    return O.macroscopic(lat, f, m, p)


def test_batch_matches_oracle_per_domain():
    doms = _domains()
    b = X.Batch(doms, OMEGA)
    b.set_masks()
    b.init()
    b.step(150)
    got = b.macroscopic()
    b.close()
    for dom, (rg, ug) in zip(doms, got):
        ro, uo = _oracle(dom, 150)
        fl = dom["mask"] == 0
        assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-4
        assert np.all(ug[:, ~fl] == 0)


def _state(b):
    return [np.concatenate([r.reshape(-1), u.reshape(-1)]) for r, u in b.macroscopic()]


def test_persistent_equals_per_domain_launches():
    doms = _domains(12, seed=3)
    a = X.Batch(doms, OMEGA)
    c = X.Batch(doms, OMEGA)
    for b in (a, c):
        b.set_masks()
        b.init()
    a.step(31)
    c.step_per_domain(31)
    for x, y in zip(_state(a), _state(c)):
        assert np.array_equal(x, y)
    a.close()
    c.close()


@pytest.mark.parametrize("threads,ctas", [(32, 1), (128, 4), (1024, 1)])
def test_launch_shapes_and_graph_replay_agree(threads, ctas):
    doms = _domains(10, seed=5)
    ref = X.Batch(doms, OMEGA)
    ref.set_masks()
    ref.init()
    ref.step(40)
    want = _state(ref)
    ref.close()
    b = X.Batch(doms, OMEGA)
    b.set_masks()
    b.init()
    X.xlb_batch_set_launch(b.b, threads, ctas)
    b.step(1)
    for _ in range(3):  # the graph of 13 steps is replayed
        b.step(13)
    for x, y in zip(_state(b), want):
        assert np.array_equal(x, y)
    b.close()


def test_tuner_picks_a_shape_and_keeps_the_state(tmp_path):
    doms = _domains(16, seed=9)
    b = X.Batch(doms, OMEGA)
    b.set_masks()
    b.init()
    b.step(7)
    before = _state(b)
    cache = str(tmp_path / "tune.json")
    th, ct = b.tune(6, cache)
    assert th in (128, 256, 512, 1024) and ct in (1, 2, 4, 8)
    assert X.xlb_batch_info(b.b)["time"] == 7
    for x, y in zip(_state(b), before):
        assert np.array_equal(x, y)
    assert b.tune(6, cache) == (th, ct)  # a cache hit
    b.close()


def test_batch_rejects_other_cell_types():
    doms = _domains(2)
    doms[1]["mask"] = doms[1]["mask"].copy()
    doms[1]["mask"][3, 3] = O.LID
    b = X.Batch(doms, OMEGA)
    with pytest.raises(X.XlbError) as e:
        b.set_masks()
    assert e.value.status == X.XLB_ERR_UNSUPPORTED
    b.close()
