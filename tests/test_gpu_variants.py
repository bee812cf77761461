"""Bulk-pass variants and the boundary tables.

The bulk variants (one cell per thread, and two or four cells per thread
with vector loads and warp shuffles) give identical populations; the
boundary tables (ghost links and inlet / outlet cells) have the sizes the
mask fixes; the 16-bit x-face links, the fix-up cells beside them and the
inflow / outflow planes that the bulk pass serves agree with the oracle;
ghost values follow changes of the lid velocity and of the mask mid-run.
"""
import numpy as np
import pytest

from oracle import lbm as O
from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X
from parity_util import Case, rel_l2

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    m = I.lid_driven_cavity_mask(32, 24, 20)
    out.append(("cavity19", Case(19, m.shape, 1.7, "bgk", mask=m, lid=(1.0, (0.05, 0.0, 0.0)))))
    sh = (40, 64)
    m = I.channel_2d_mask(64, 40, top=O.LID)
    m[I.random_obstacle_mask(sh, 0.06, seed=3) > 0] = O.WALL
    m[I.random_obstacle_mask(sh, 0.02, seed=4) > 0] = O.EQ
    r, u = I.random_flow(sh, 2, seed=5, rho_amp=0.005, u_amp=0.02)
    out.append(("mixed9", Case(9, sh, 1.3, "bgk", mask=m, force=(1e-5, 2e-6, 0.0),
                               lid=(1.0, (0.03, 0.0, 0.0)), eq=(1.0, (0.01, 0.0, 0.0)), rho0=r, u0=u)))
    r, u = I.random_flow((8, 12, 48), 3, seed=6, rho_amp=0.01, u_amp=0.03)
    out.append(("periodic27", Case(27, (8, 12, 48), 1.5, "bgk", rho0=r, u0=u)))
    m = I.lid_driven_cavity_mask(72, 10, 12)  # 72 / 4 = 18 slots: partial warps
    out.append(("ragged19", Case(19, m.shape, 1.7, "bgk", mask=m, lid=(1.0, (0.05, 0.0, 0.0)))))
    m = I.channel_2d_mask(64, 40)  # WALL faces; FWALL obstacles are fix-up cells
    m[I.random_obstacle_mask(sh, 0.05, seed=7) > 0] = O.FWALL
    m[0, :] = O.WALL
    m[-1, :] = O.WALL
    r, u = I.random_flow(sh, 2, seed=8, rho_amp=0.005, u_amp=0.02)
    out.append(("fwall9", Case(9, sh, 1.4, "bgk", mask=m, force=(1e-5, 0.0, 0.0), rho0=r, u0=u)))
    # x-face planes of the other two types: EQ at x = 0, a tangentially moving
    # LID at x = nx - 1, meeting WALL rows; interior obstacles, some beside
    # the x-faces
    sh = (36, 64)
    m = np.zeros(sh, np.uint8)
    m[:, 0] = O.EQ
    m[:, -1] = O.LID
    m[0, :] = O.WALL
    m[-1, :] = O.WALL
    obst = I.random_obstacle_mask(sh, 0.05, seed=11) > 0
    obst[[0, -1], :] = False
    obst[:, [0, -1]] = False
    m[obst] = O.WALL
    r, u = I.random_flow(sh, 2, seed=12, rho_amp=0.005, u_amp=0.02)
    out.append(("xfaces9", Case(9, sh, 1.5, "bgk", mask=m, force=(0.0, 1e-5, 0.0), lid=(1.0, (0.0, 0.03, 0.0)),
                                eq=(1.0, (0.02, 0.01, 0.0)), rho0=r, u0=u)))
    # inflow / outflow planes served by the bulk pass: D2Q9 channel, INLET
    # column x = 0 (Zou-He), OUTLET column x = nx - 1, WALL rows, obstacles
    sh = (34, 96)
    m = I.channel_2d_mask(96, 34)
    m[1:-1, 0] = O.INLET
    m[1:-1, -1] = O.OUTLET
    obst = I.random_obstacle_mask(sh, 0.03, seed=16) > 0
    obst[[0, -1], :] = False
    obst[:, [0, 1, -2, -1]] = False
    m[obst] = O.WALL
    r, u = I.random_flow(sh, 2, seed=17, rho_amp=0.005, u_amp=0.02)
    out.append(("inout9", Case(9, sh, 1.5, "bgk", mask=m, inlet=(0.03, 0.0, 0.0), rho0=r, u0=u)))
    # the same in 3D: D3Q19 channel, WALL y faces (so the outlet's copied
    # directions meet face rules), periodic in z, INLET / OUTLET planes
    m = np.zeros((10, 12, 48), np.uint8)
    m[:, 0, :] = O.WALL
    m[:, -1, :] = O.WALL
    m[:, 1:-1, 0] = O.INLET
    m[:, 1:-1, -1] = O.OUTLET
    m[4:6, 5:7, 20:23] = O.WALL
    r, u = I.random_flow(m.shape, 3, seed=18, rho_amp=0.005, u_amp=0.02)
    out.append(("inout19", Case(19, m.shape, 1.6, "bgk", mask=m, inlet=(0.03, 0.0, 0.0), rho0=r, u0=u)))
    # D3Q19: EQ x = 0 face, LID x = nx - 1 face moving along z, WALL y faces,
    # periodic in z; 40 / 4 = 10 slots per row (a partial warp)
    m = np.zeros((10, 12, 40), np.uint8)
    m[:, :, 0] = O.EQ
    m[:, :, -1] = O.LID
    m[:, 0, :] = O.WALL
    m[:, -1, :] = O.WALL
    r, u = I.random_flow(m.shape, 3, seed=13, rho_amp=0.005, u_amp=0.02)
    out.append(("xfaces19", Case(19, m.shape, 1.6, "bgk", mask=m, lid=(1.0, (0.0, 0.0, 0.03)),
                                 eq=(1.0, (0.02, 0.0, 0.01)), rho0=r, u0=u)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("variant", ["vec", "vec2"])
def test_vec_equals_direct(name, case, storage, variant):
    if case.q == 27:
        pytest.skip("the vectorised kernel covers D2Q9 / D3Q19")
    a = case.gpu_sim(storage, "direct")
    b = case.gpu_sim(storage, variant)
    want = X.XLB_KERNEL_VEC if variant == "vec" else X.XLB_KERNEL_VEC2
    assert a.kernel() == X.XLB_KERNEL_DIRECT and b.kernel() == want
    a.step(40)
    b.step(40)
    pa, _ = a.populations()
    pb, _ = b.populations()
    fl = O.fluid_like(case.mask)
    assert np.array_equal(pa[:, fl], pb[:, fl])
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_switching_variants_mid_run_is_exact(storage):
    """Every bulk variant leaves the same ghost values in the boundary faces,
    so switching variants between steps changes nothing."""
    name, case = CASES[0]  # the cavity: WALL and LID faces
    a = case.gpu_sim(storage, "direct")
    b = case.gpu_sim(storage, "direct")
    a.step(60)
    b.step(20)
    b.set_kernel("vec")
    b.step(20)
    b.set_kernel("vec2")
    b.step(10)
    b.set_kernel("direct")
    b.step(10)
    pa, _ = a.populations()
    pb, _ = b.populations()
    fl = O.fluid_like(case.mask)
    assert np.array_equal(pa[:, fl], pb[:, fl])
    a.close()
    b.close()


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_vec_f16_matches_oracle(name, case):
    if case.q == 27:
        pytest.skip("the vectorised kernel covers D2Q9 / D3Q19")
    (rho_o, u_o), _ = case.oracle(120)
    rho_g, u_g = case.gpu(120, "f16", "vec")
    fl = O.fluid_like(case.mask)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= 5e-3


def test_auto_picks_the_variant_by_storage():
    """AUTO: FP16 runs 4 cells per thread without boundary planes and 2 with
    them; BF16 and FP32 one cell per thread; VEC needs 16-bit storage."""
    m = I.lid_driven_cavity_mask(32, 8, 8)
    c = Case(19, m.shape, 1.5, "bgk", mask=m)
    s32 = c.gpu_sim("f32")
    s16 = c.gpu_sim("f16")
    sb16 = c.gpu_sim("bf16")
    assert s32.kernel() == X.XLB_KERNEL_DIRECT
    assert s16.kernel() == X.XLB_KERNEL_VEC2  # the cavity's walls
    assert sb16.kernel() == X.XLB_KERNEL_DIRECT
    per16 = Case(19, (8, 8, 32), 1.5, "bgk").gpu_sim("f16")
    assert per16.kernel() == X.XLB_KERNEL_VEC
    with pytest.raises(X.XlbError) as e:
        X.xlb_set_kernel(s32.ctx, X.XLB_KERNEL_VEC)
    assert e.value.status == X.XLB_ERR_UNSUPPORTED
    odd = Case(9, (30, 45), 1.2).gpu_sim("f16")
    assert odd.kernel() == X.XLB_KERNEL_DIRECT  # nx odd
    for s in (s32, s16, sb16, odd, per16):
        s.close()


def _one_x_face_cavity():
    """The cavity with its x = nx - 1 plane opened (fluid inside the y / z
    face planes, the lid running through to the edge): only the x = 0 face
    remains."""
    m = I.lid_driven_cavity_mask(20, 18, 16)
    m[1:-1, 1:-1, -1] = O.FLUID
    m[-1, 1:-1, -1] = O.LID
    return m


def test_16_bit_x_faces_are_served_by_ghost_links():
    """With 16-bit storage the sources on WALL / LID / EQ x-face planes are
    ghost links (the bulk pass then runs no face logic at the ends of a row);
    the y / z faces stay faces.  FP32 keeps all six faces."""
    yz = [(1, 0), (1, -1), (0, 0), (0, -1)]
    m20 = I.lid_driven_cavity_mask(20, 18, 16)
    m33 = I.lid_driven_cavity_mask(33, 10, 9)
    one = _one_x_face_cavity()
    w32_one = _links(19, one, yz + [(2, 0)])  # FP32: the x = 0 face stays a face
    for m, w32 in ((m20, 0), (m33, 0), (one, w32_one)):
        w16 = _links(19, m, yz)
        assert w16 > 0
        for st in ("f32", "f16", "bf16"):
            s = X.Simulation(19, tuple(reversed(m.shape)), 1.5, "bgk", st)
            s.set_mask(m)
            assert X.xlb_boundary_links(s.ctx) == (w32 if st == "f32" else w16, 0), (m.shape, st)
            s.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("kind", ["nx33", "one_face"])
def test_linked_x_faces_match_oracle(storage, kind):
    """The ghost links of the 16-bit x-faces with an odd nx (one cell per
    thread) and with a single x-face, against the oracle, at the storage
    bound."""
    m = I.lid_driven_cavity_mask(33, 10, 9) if kind == "nx33" else _one_x_face_cavity()
    r, u = I.random_flow(m.shape, 3, seed=14, rho_amp=0.005, u_amp=0.02)
    c = Case(19, m.shape, 1.6, "bgk", mask=m, lid=(1.0, (0.05, 0.0, 0.0)), rho0=r, u0=u)
    (_, u_o), _ = c.oracle(100)
    _, u_g = c.gpu(100, storage)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= 5e-3


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_inlet_cells_beside_x_faces(storage):
    """INLET and OUTLET segments in the columns next to WALL x-faces (fix-up
    cells, whose boundary links sit beside the x-face ghost links of the
    fluid cells around the segments), against the oracle."""
    sh = (40, 64)
    m = I.channel_2d_mask(64, 40)
    m[:, 0] = O.WALL
    m[:, -1] = O.WALL
    m[12:25, 1] = O.INLET
    m[8:30, -2] = O.OUTLET
    r, u = I.random_flow(sh, 2, seed=15, rho_amp=0.005, u_amp=0.02)
    c = Case(9, sh, 1.5, "bgk", mask=m, inlet=(0.03, 0.0, 0.0), rho0=r, u0=u)
    (_, u_o), _ = c.oracle(150)
    _, u_g = c.gpu(150, storage)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= (1e-4 if storage == "f32" else 5e-3)


def _links(q, m, skip_faces=(), io_owners=False, owner_mask=None):
    """Ghost links: (owner cell, direction) with a WALL / LID / EQ source off
    the listed face planes; owners are FLUID cells and, with io_owners, the
    inflow / outflow cells the bulk pass serves (owner_mask, else all INLET
    and OUTLET cells)."""
    lat = O.Lattice(q)
    owners = m == O.FLUID
    if io_owners:
        owners = owners | (owner_mask if owner_mask is not None else np.isin(m, (O.INLET, O.OUTLET)))
    n = 0
    for i in range(1, q):
        src_nonfluid = ~O.fluid_like(lat.roll(m, i))
        on_face = np.zeros(m.shape, bool)
        for ax, side in skip_faces:  # ax in array-axis order, side 0 / -1
            idx = [slice(None)] * m.ndim
            coord = np.arange(m.shape[ax])
            shift = int(lat.c[i][::-1][ax])
            src_coord = (coord - shift) % m.shape[ax]
            hit = src_coord == (0 if side == 0 else m.shape[ax] - 1)
            sh = [1] * m.ndim
            sh[ax] = m.shape[ax]
            on_face |= hit.reshape(sh)
        n += int((owners & src_nonfluid & ~on_face).sum())
    return n


def test_boundary_tables():
    """Ghost links: one per (fluid cell, direction) whose source is WALL, LID
    or EQ and not on a boundary face plane the mask fills uniformly (those the
    pull handles by coordinates); one fix-up entry per inlet / outlet cell."""
    cav = I.lid_driven_cavity_mask(20, 18, 16)
    holed = cav.copy()
    holed[5:8, 6:9, 0] = O.FLUID  # x = 0 plane no longer a face
    sph = I.sphere_channel_mask(40, 16, 12, radius=3, center=(12, 8, 6))
    eqs = np.where(I.random_obstacle_mask((30, 40), 0.1, seed=2) > 0, O.EQ, 0).astype(np.uint8)
    all_faces = [(2, 0), (2, -1), (1, 0), (1, -1), (0, 0), (0, -1)]
    # the hole removes the x = 0 face; the lid plane's x = 0 edge cells are
    # WALL, which only the x = 0 face explained, so the lid face goes too
    holed_faces = [f for f in all_faces if f not in ((2, 0), (0, -1))]
    seg = I.channel_2d_mask(40, 30)
    seg[10:20, 0] = O.INLET  # a segment: its cells stay fix-up cells
    seg[1:-1, -1] = O.OUTLET
    seg[12:15, 1:3] = O.WALL  # an obstacle touching the inlet segment
    for q, m, faces, planes in ((19, cav, all_faces, False), (19, holed, holed_faces, False),
                                (27, sph, [], True), (9, eqs, [], False), (9, seg, [(0, 0), (0, -1)], False)):
        # the whole INLET plane x = 0 / OUTLET plane x = nx - 1 of the sphere
        # channel is served by the bulk pass: no fix-up cells, links owned
        io = np.isin(m, (O.INLET, O.OUTLET))
        want = (_links(q, m, faces, io_owners=planes), 0 if planes else int(io.sum()))
        if m is seg:  # the outlet column is a whole plane, the inlet segment is not
            want = (_links(q, m, faces, io_owners=True, owner_mask=(m == O.OUTLET)), int((m == O.INLET).sum()))
        s = X.Simulation(q, tuple(reversed(m.shape)), 1.5, "bgk")
        s.set_mask(m)
        assert X.xlb_boundary_links(s.ctx) == want, (m.shape, want)
        s.close()
    assert _links(19, cav, all_faces) == 0


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_faces_and_ghosts_mixed_parity(storage):
    """A cavity whose x = 0 wall has a hole (no longer a face: ghost links),
    an EQ top face, interior obstacles: against the oracle."""
    m = I.lid_driven_cavity_mask(32, 20, 18)
    m[m == O.LID] = O.EQ
    m[6:10, 5:9, 0] = O.FLUID
    m[I.random_obstacle_mask(m.shape, 0.03, seed=9) > 0] = O.WALL
    rho, u = I.random_flow(m.shape, 3, seed=10, rho_amp=0.005, u_amp=0.02)
    c = Case(19, m.shape, 1.6, "bgk", mask=m, eq=(1.0, (0.03, 0.0, 0.0)), rho0=rho, u0=u)
    (rho_o, u_o), _ = c.oracle(100)
    rho_g, u_g = c.gpu(100, storage)
    fl = O.fluid_like(m)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= (1e-4 if storage == "f32" else 5e-3)


def test_ghosts_follow_lid_and_mask_changes():
    """Changing the lid velocity or the mask between steps takes effect at
    the next step exactly as in the oracle (the ghost values are refreshed)."""
    m1 = I.channel_2d_mask(48, 20, top=O.LID)
    m2 = m1.copy()
    m2[8:12, 20:24] = O.WALL
    c = Case(9, m1.shape, 1.4, "bgk", mask=m1, lid=(1.0, (0.04, 0.0, 0.0)))
    sim = c.gpu_sim()
    sim.step(30)
    sim.set_bc(X.XLB_CELL_LID, 1.0, (-0.02, 0.01, 0.0))
    sim.step(30)
    sim.set_mask(m2)
    sim.step(30)
    _, ug = sim.macroscopic()
    sim.close()
    lat = c.lat
    p = c.params()
    f = O.run(lat, O.init_state(lat, c.rho0, c.u0, m1, p), m1, p, 30)
    p.bc.lid_u = [-0.02, 0.01]
    f = O.run(lat, f, m1, p, 30)
    f = O.run(lat, f, m2, p, 30)
    _, uo = O.macroscopic(lat, f, m2, p)
    fl = O.fluid_like(m2)
    assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-4


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_inflow_outflow_planes_match_oracle(storage):
    """Whole INLET / OUTLET x-planes served by the bulk pass (no fix-up
    cells), D3Q19 with WALL y faces meeting them and an obstacle; the
    regularized inlet; against the oracle."""
    name, case = [c for c in CASES if c[0] == "inout19"][0]
    c = Case(case.q, case.shape, case.omega, "bgk", mask=case.mask, inlet=case.inlet, rho0=case.rho0, u0=case.u0,
             inlet_scheme="regularized")
    sim = c.gpu_sim(storage)
    assert X.xlb_boundary_links(sim.ctx)[1] == 0
    sim.close()
    (_, u_o), _ = c.oracle(120)
    _, u_g = c.gpu(120, storage)
    fl = O.fluid_like(c.mask)
    assert rel_l2(u_g[:, fl], u_o[:, fl]) <= (1e-4 if storage == "f32" else 5e-3)
