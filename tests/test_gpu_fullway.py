"""Full-way bounce-back walls (FWALL) and the performance cavity of
Section 5 (FWALL walls, equilibrium-BC lid) on the GPU, against the FP64
oracle.

FWALL cells on whole face planes are reversed by the bulk kernel by their
coordinates; FWALL cells elsewhere (obstacles, a wall plane with a hole) go
through the fix-up list.  Both are compared with the oracle; stream-only runs
are bit-exact.  Tolerances as in the other parity tests: FP32 u rel-L2
<= 1e-4, FP16 and BF16 <= 5e-3.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import Case, f64_to_raw, raw_to_f64, rel_l2, storage_dtype

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f16": 5e-3, "bf16": 5e-3}
EQ_LID = (1.0, (0.05, 0.0, 0.0))


def _start(shape, d, seed):
    rho, u = I.random_flow(shape, d, seed=seed, rho_amp=0.005, u_amp=0.02)
    return rho.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_paper_cavity_d3q19(storage):
    """The Section 5 cavity on a non-cubic box (faces on every plane)."""
    m = I.paper_cavity_mask(26, 22, 20)
    rho, u = _start(m.shape, 3, 3)
    c = Case(19, m.shape, 1.7, "bgk", mask=m, eq=EQ_LID, rho0=rho, u0=u)
    (_, u_o), _ = c.oracle(150)
    _, u_g = c.gpu(150, storage)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= TOL[storage]
    assert np.all(u_g[:, m == O.FWALL] == 0.0)


def test_paper_cavity_kbc_d3q27():
    m = I.paper_cavity_mask(20, 18, 16)
    rho, u = _start(m.shape, 3, 4)
    c = Case(27, m.shape, 1.9, "kbc", mask=m, eq=EQ_LID, rho0=rho, u0=u)
    (_, u_o), _ = c.oracle(120)
    _, u_g = c.gpu(120)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= 1e-4


def _holed_cavity():
    """Section 5 cavity whose x = 0 FWALL plane has a hole (no longer a face:
    its FWALL cells become fix-up cells, and the EQ lid plane, whose x = 0 edge
    only that face explained, falls back to ghost links), plus FWALL and WALL
    obstacles, some of them touching each other."""
    m = I.paper_cavity_mask(30, 20, 18)
    m[7:10, 6:9, 0] = O.FLUID
    inner = np.zeros(m.shape, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    m[inner & (I.random_obstacle_mask(m.shape, 0.03, seed=21) > 0)] = O.FWALL
    m[inner & (I.random_obstacle_mask(m.shape, 0.03, seed=22) > 0)] = O.WALL
    m[5:8, 8:11, 12:15] = O.FWALL
    m[6, 9, 15] = O.WALL
    return m


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_fullway_obstacles_and_holed_face(storage):
    m = _holed_cavity()
    rho, u = _start(m.shape, 3, 5)
    c = Case(19, m.shape, 1.5, "bgk", mask=m, eq=EQ_LID, force=(2e-6, 0.0, 1e-6), rho0=rho, u0=u)
    (_, u_o), _ = c.oracle(120)
    _, u_g = c.gpu(120, storage)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= TOL[storage]


@pytest.mark.parametrize("collision", ["bgk", "kbc"])
def test_fullway_d2q9_channel(collision):
    """D2Q9 channel: FWALL bottom face, moving halfway LID on top, FWALL and
    WALL obstacles (an FWALL cell next to a WALL cell pulls its ghost)."""
    m = I.channel_2d_mask(70, 30, top=O.LID, bottom=O.FWALL)
    m[I.random_obstacle_mask(m.shape, 0.04, seed=31) > 0] = O.FWALL
    m[I.random_obstacle_mask(m.shape, 0.02, seed=32) > 0] = O.WALL
    m[0, :] = O.FWALL
    m[29, :] = O.LID
    m[10:13, 20:23] = O.FWALL
    m[11, 23] = O.WALL
    rho, u = _start(m.shape, 2, 6)
    c = Case(9, m.shape, 1.6, collision, mask=m, lid=(1.0, (0.04, 0.0, 0.0)), rho0=rho, u0=u)
    (_, u_o), _ = c.oracle(300)
    _, u_g = c.gpu(300)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= 1e-4


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_fullway_stream_only_is_bit_exact(storage):
    """Collision NONE leaves FWALL cells unreversed: n steps permute the
    populations of the fluid and FWALL cells (WALL sources bounce back),
    bit for bit, with FWALL faces, FWALL fix-up cells and WALL ghosts."""
    shape = (12, 10, 16)
    m = np.zeros(shape, np.uint8)
    m[:, :, 0] = O.FWALL
    m[:, :, -1] = O.FWALL
    m[0, :, :] = O.WALL
    m[I.random_obstacle_mask(shape, 0.05, seed=41) > 0] = O.FWALL
    m[I.random_obstacle_mask(shape, 0.03, seed=42) > 0] = O.WALL
    lat = O.Lattice(19)
    sim = X.Simulation(19, tuple(reversed(shape)), 1.0, "none", storage)
    sim.set_mask(m)
    sim.init()
    rng = np.random.default_rng(43)
    vals = rng.uniform(-0.05, 0.05, (19,) + shape)
    if storage == "bf16":
        raw = (vals.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    else:
        raw = vals.astype(storage_dtype(storage))
    buf = sim.state_get().copy()
    buf[:64].view(np.int32)[12] = 1
    data = buf[64:].view(raw.dtype)
    align = 256 // raw.itemsize
    plane = (sim.N + align - 1) // align * align
    data.reshape(19, plane)[:, :sim.N] = raw.reshape(19, sim.N)
    sim.state_set(buf)
    n = 6
    sim.step(n)
    got, kind = sim.populations()
    assert kind == 1
    # at the cells that hold state every pulled value is a copy (plain, or
    # bounced back from a WALL source), so the oracle's stream can act on the
    # stored deviations directly
    h = raw_to_f64(raw, storage)
    for _ in range(n):
        h = O.stream_bc(lat, h, m, O.BC(3))
    held = (m == O.FLUID) | (m == O.FWALL)
    want = np.ascontiguousarray(f64_to_raw(h[:, held], storage))
    assert np.array_equal(np.ascontiguousarray(got[:, held]).view(np.uint8), want.view(np.uint8))
    sim.close()


def _face_planes(m, faces):
    on = np.zeros(m.shape, bool)
    for ax, pos in faces:
        sl = [slice(None)] * m.ndim
        sl[ax] = pos
        on[tuple(sl)] = True
    return on


def _expected_tables(q, m, faces):
    """(n_links, n_fix) written out from the definition of the tables."""
    lat = O.Lattice(q)
    on = _face_planes(m, faces)
    owner = (m == O.FLUID) | ((m == O.FWALL) & on)
    n = 0
    for i in range(1, q):
        src = lat.roll(m, i)
        src_on = lat.roll(on.astype(np.uint8), i).astype(bool)
        ghost = np.isin(src, (O.WALL, O.LID, O.EQ)) & ~src_on
        n += int((owner & ghost).sum())
    fix = int(np.isin(m, (O.INLET, O.OUTLET)).sum()) + int(((m == O.FWALL) & ~on).sum())
    return n, fix


def test_fullway_boundary_tables():
    cav = I.paper_cavity_mask(20, 18, 16)
    all_faces = [(2, 0), (2, -1), (1, 0), (1, -1), (0, 0), (0, -1)]
    holed = _holed_cavity()
    # the hole drops the x = 0 face and, with it, the EQ lid face
    holed_faces = [(2, -1), (1, 0), (1, -1), (0, 0)]
    for m, faces in ((cav, all_faces), (holed, holed_faces)):
        s = X.Simulation(19, tuple(reversed(m.shape)), 1.5, "bgk")
        s.set_mask(m)
        assert X.xlb_boundary_links(s.ctx) == _expected_tables(19, m, faces)
        s.close()
    assert _expected_tables(19, cav, all_faces) == (0, 0)


def test_fullway_mask_change_mid_run():
    """FWALL obstacles added between steps act from the next step on, as in
    the oracle (the first update after the change collides locally, which
    reverses the new FWALL cells)."""
    m1 = I.paper_cavity_mask(28, 18, 16)
    m2 = m1.copy()
    m2[6:9, 7:10, 10:13] = O.FWALL
    rho, u = _start(m1.shape, 3, 7)
    c = Case(19, m1.shape, 1.4, "bgk", mask=m1, eq=EQ_LID, rho0=rho, u0=u)
    sim = c.gpu_sim()
    sim.step(40)
    sim.set_mask(m2)
    sim.step(40)
    _, u_g = sim.macroscopic()
    sim.close()
    lat, p = c.lat, c.params()
    f = O.run(lat, O.init_state(lat, c.rho0, c.u0, m1, p), m1, p, 40)
    f = O.run(lat, f, m2, p, 40)
    _, u_o = O.macroscopic(lat, f, m2, p)
    fl = O.fluid_like(m2)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= 1e-4


def test_fullway_kernel_choice_and_adjoint():
    """A mask with FWALL faces runs the one-cell kernel even when the
    vectorised one is requested, and the adjoint refuses FWALL cells."""
    m = I.paper_cavity_mask(32, 16, 16)
    s = X.Simulation(19, (32, 16, 16), 1.5, "bgk", "f16")
    s.set_kernel("vec")
    s.set_mask(m)
    assert s.kernel() == X.XLB_KERNEL_DIRECT
    s.close()
    s = X.Simulation(19, (32, 16, 16), 1.5, "bgk", "f32")
    s.set_mask(m)
    s.init()
    with pytest.raises(X.XlbError):
        X.xlb_tape_begin(s.ctx, 4, 2)
    s.close()


def test_full_size_paper_cavity_sampled_step():
    """256^3 Section 5 cavity in the benchmark's configuration: after some
    steps, one more GPU step is checked cell by cell on a sample (interior,
    next to the walls and the lid, on the FWALL faces and edges, on the lid)
    against the oracle's C(S_bc(.)) on each cell's periodic 3x3x3
    neighbourhood."""
    n = 256
    mask = I.paper_cavity_mask(n)
    nu = 0.05 * (n - 2) / 1000.0
    omega = X.xlb_omega_from_nu(nu)
    c = Case(19, mask.shape, omega, "bgk", mask=mask, eq=EQ_LID)
    sim = c.gpu_sim()
    sim.step(30)
    h_prev, k1 = sim.populations()
    sim.step(1)
    h_next, k2 = sim.populations()
    assert k1 == 1 and k2 == 1
    rng = np.random.default_rng(1)
    pts = [tuple(rng.integers(1, n - 1, 3)) for _ in range(200)]
    pts += [(z, y, x) for z in (0, 1, n - 2) for y in (0, 1, 2, n - 2, n - 1) for x in (0, 1, 5, n - 2, n - 1)]
    lat = c.lat
    p = c.params()
    w = lat.w[:, None, None, None]
    worst = 0.0
    for (z, y, x) in pts:
        idx = np.ix_([(z + d) % n for d in (-1, 0, 1)], [(y + d) % n for d in (-1, 0, 1)],
                     [(x + d) % n for d in (-1, 0, 1)])
        mp = mask[idx]
        if mp[1, 1, 1] not in (O.FLUID, O.FWALL):
            continue
        hp = h_prev[(slice(None),) + idx].astype(np.float64) + w
        f = O.stream_bc(lat, hp, mp, p.bc)
        hn = O.collide(lat, f, mp, p)[:, 1, 1, 1] - lat.w
        g = h_next[:, z, y, x].astype(np.float64)
        worst = max(worst, float(np.max(np.abs(g - hn))))
    assert worst < 2e-7
    sim.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_inflow_outflow_columns_with_fwall_faces(storage):
    """A D2Q9 channel with FWALL rows as faces and whole INLET / OUTLET
    columns: with an FWALL face the bulk pass does not serve the columns, so
    they stay fix-up cells; against the oracle."""
    m = I.channel_2d_mask(64, 26, top=O.FWALL, bottom=O.FWALL)
    m[1:-1, 0] = O.INLET
    m[1:-1, -1] = O.OUTLET
    rho, u = _start(m.shape, 2, 9)
    c = Case(9, m.shape, 1.5, "bgk", mask=m, inlet=(0.03, 0.0, 0.0), rho0=rho, u0=u)
    sim = c.gpu_sim(storage)
    assert X.xlb_boundary_links(sim.ctx) == (0, 2 * 24)
    sim.close()
    (_, u_o), _ = c.oracle(150)
    _, u_g = c.gpu(150, storage)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= TOL[storage]
