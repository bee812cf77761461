"""Seeded synthetic workloads shared by the tests, the benchmark and smoke().

This module builds inputs only: cell-type masks, initial density / velocity
fields and batch descriptors.  It holds no lattice Boltzmann arithmetic (no
equilibrium, collision, streaming or boundary rule), so the CUDA path and the
CPU oracle can both consume its arrays without sharing any of the method.

Array layout is the library's: 3D fields are ``[z, y, x]`` and 2D fields
``[y, x]`` (x fastest); vector fields put the component first (``u[a, ...]``).
The mask codes are the cell types of the C ABI (``include/xlb.h``).
"""
from __future__ import annotations

import numpy as np

FLUID, WALL, LID, INLET, OUTLET, EQ, FWALL = 0, 1, 2, 3, 4, 5, 6


def taylor_green_2d(nx, ny, u0=0.04, rho0=1.0):
    """Initial fields of the 2D Taylor-Green vortex (Section 4.1, Eq. 9, t = 0).

    Cell centres sit at integer coordinates; k = 2 pi / n.  The density carries
    the pressure perturbation through p = cs^2 rho (Eq. 8):
    rho = rho0 - (3 rho0 u0^2 / 4) [cos 2 kx x + cos 2 ky y].
    """
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    ux = u0 * np.sin(kx * x) * np.cos(ky * y)
    uy = -u0 * np.cos(kx * x) * np.sin(ky * y)
    rho = rho0 - 0.75 * rho0 * u0 * u0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    return rho, np.stack([ux, uy])


def taylor_green_amplitude_factor(t, nu, nx, ny):
    """Velocity decay factor exp(-nu (kx^2 + ky^2) t) of the Taylor-Green
    vortex (Section 4.1, Eq. 9).  The paper prints t_d = [2 nu (kx^2+ky^2)]^-1
    with exp(-t/t_d); the Navier-Stokes solution it states decays at half that
    rate, so the velocity factor here uses t_d = [nu (kx^2 + ky^2)]^-1."""
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    return float(np.exp(-t * nu * (kx * kx + ky * ky)))


def lid_driven_cavity_mask(n, ny=None, nz=None):
    """Cubic cavity (Section 4.2): the six boundary planes are solid; the top
    plane z = nz-1 is the moving LID, the other five planes are WALL, and edges
    and corners shared with a side wall are WALL."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[nz - 1, :, :] = LID
    m[0, :, :] = WALL
    m[:, 0, :] = WALL
    m[:, ny - 1, :] = WALL
    m[:, :, 0] = WALL
    m[:, :, nx - 1] = WALL
    return m


def paper_cavity_mask(n, ny=None, nz=None):
    """The cavity of the paper's performance runs (Section 5): full-way
    bounce-back walls (FWALL) on five faces and an equilibrium-BC lid (EQ) on
    the top plane z = nz-1, whose edges shared with a wall are FWALL."""
    m = lid_driven_cavity_mask(n, ny, nz)
    m[m == WALL] = FWALL
    m[m == LID] = EQ
    return m


def sphere_channel_mask(nx, ny, nz, radius, center=None):
    """Channel along x with a solid sphere (config "flow past a sphere"):
    INLET plane x = 0, OUTLET plane x = nx-1, periodic in y and z; cell (i, j, k)
    is WALL iff (i-cx)^2 + (j-cy)^2 + (k-cz)^2 <= r^2."""
    if center is None:
        center = (nx // 4, ny // 2, nz // 2)
    cx, cy, cz = center
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[(x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= radius * radius] = WALL
    m[:, :, 0] = INLET
    m[:, :, nx - 1] = OUTLET
    return m


def schafer_turek_2d(n_d, u_mean):
    """The 2D flow-around-a-cylinder benchmark of Schafer and Turek (1996)
    that Section 4.3 uses: channel 2.2 x 0.41, cylinder of diameter D = 0.1
    centred at (0.2, 0.2), parabolic inflow of mean speed U; n_d cells per D.

    Cells: WALL rows y = 0 and ny - 1 (no-slip lines half a cell inside, at
    y = 1/2 and ny - 3/2, so the channel is H = 4.1 n_d cells high), INLET
    column x = 0, OUTLET column x = nx - 1 = 22 n_d, cylinder cells WALL where
    the cell centre lies within D/2 of (2 n_d, 2 n_d + 1/2).
    Returns (mask[ny, nx], center (x, y), radius, inlet velocity field
    u[2, ny, nx] = (4 U_m y' (H - y') / H^2, 0) with y' = y - 1/2 and
    U_m = 3 U / 2)."""
    H = round(4.1 * n_d)
    ny, nx = H + 2, 22 * n_d + 1
    center = (2.0 * n_d, 2.0 * n_d + 0.5)
    radius = 0.5 * n_d
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    m = np.zeros((ny, nx), dtype=np.uint8)
    m[(x - center[0]) ** 2 + (y - center[1]) ** 2 <= radius * radius] = WALL
    m[1:ny - 1, 0] = INLET
    m[1:ny - 1, nx - 1] = OUTLET
    m[0, :] = WALL
    m[ny - 1, :] = WALL
    yp = np.arange(ny) - 0.5
    prof = 4.0 * 1.5 * u_mean * yp * (H - yp) / (H * H)
    prof[0] = prof[ny - 1] = 0.0
    u = np.zeros((2, ny, nx))
    u[0] = prof[:, None]
    return m, center, radius, u


def ball_links(mask, center, radius, c):
    """Links from FLUID cells to the cells of a disc / ball (cell centres
    within `radius` of `center` = (x, y[, z])), with the fraction q in [0, 1]
    of each link at which it enters the circle / sphere.  c: the lattice
    velocities (Q x d, Figure 1 order).  Returns (cells as flat indices, x
    fastest; directions; q)."""
    d = mask.ndim
    c = np.asarray(c)
    coords = np.meshgrid(*[np.arange(n) for n in mask.shape], indexing="ij")
    pos = [coords[d - 1 - a] for a in range(d)]          # x, y[, z]
    ctr = np.asarray(center, dtype=float)
    inside = sum((pos[a] - ctr[a]) ** 2 for a in range(d)) <= radius * radius
    cells, dirs, qs = [], [], []
    fl = np.argwhere(mask == FLUID)
    for i in range(1, c.shape[0]):
        ci = c[i, :d]
        tgt = fl[:, ::-1] + ci                            # (x, y[, z]) of x + c_i
        ok = np.all((tgt >= 0) & (tgt < np.array(mask.shape[::-1])), axis=1)
        src, tgt = fl[ok], tgt[ok]
        hit = inside[tuple(tgt[:, ::-1].T)] & (mask[tuple(tgt[:, ::-1].T)] == WALL)
        src = src[hit]
        if not len(src):
            continue
        r0 = src[:, ::-1].astype(float) - ctr                 # x - C
        a = float(ci @ ci)
        b = 2.0 * (r0 @ ci)
        cc = (r0 * r0).sum(axis=1) - radius * radius
        t = (-b - np.sqrt(np.maximum(b * b - 4.0 * a * cc, 0.0))) / (2.0 * a)
        t = np.clip(t, 0.0, 1.0)   # a cell centre on the surface gives q = 0 up to rounding
        cells.append(np.ravel_multi_index(tuple(src.T), mask.shape))
        dirs.append(np.full(len(src), i))
        qs.append(t)
    if not cells:
        return np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0)
    return np.concatenate(cells).astype(np.int64), np.concatenate(dirs).astype(np.int32), np.concatenate(qs)


def channel_2d_mask(nx, ny, top=WALL, bottom=WALL):
    """2D channel periodic in x with solid rows y = 0 and y = ny-1."""
    m = np.zeros((ny, nx), dtype=np.uint8)
    m[0, :] = bottom
    m[ny - 1, :] = top
    return m


def density_perturbation(shape, amplitude=1e-3, seed=1234):
    """i.i.d. Gaussian density perturbation N(0, 1) * amplitude (seeded)."""
    rng = np.random.default_rng(seed)
    return amplitude * rng.standard_normal(shape)


def random_flow(shape, d, seed, rho_amp=1e-2, u_amp=0.03):
    """Smooth-ish random initial fields for parity tests: rho = 1 + noise,
    |u| up to ``u_amp`` per component (uniform), seeded."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, size=shape)
    u = u_amp * rng.uniform(-1, 1, size=(d,) + tuple(shape))
    return rho, u


def random_obstacle_mask(shape, fraction, seed, code=WALL):
    """Scattered solid cells (for bounce-back parity on irregular geometry)."""
    rng = np.random.default_rng(seed)
    m = np.zeros(shape, dtype=np.uint8)
    m[rng.random(shape) < fraction] = code
    return m


def batched_channels(n_domains, seed=1234, nx_range=(32, 256), ny_range=(32, 128),
                     n_obstacles=(1, 5), radius=(3, 12), nu=0.1, u_max=0.05):
    """Batch of independent 2D channels (config "batched channel flows").

    Each domain: nx ~ U{nx_range}, ny ~ U{ny_range}; WALL rows y = 0 and
    y = ny-1; periodic in x; 1-5 solid discs with radius 3-12 at seeded centres
    inside the fluid; body force F_x = 8 nu u_max / H^2 with H = ny - 2.
    One child seed per domain from the master seed.
    Returns a list of dicts {nx, ny, mask[ny, nx] uint8, force (Fx, 0)}.
    """
    master = np.random.default_rng(seed)
    seeds = master.integers(0, 2 ** 63 - 1, size=n_domains)
    out = []
    for s in seeds:
        rng = np.random.default_rng(int(s))
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        m = channel_2d_mask(nx, ny)
        y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        k = int(rng.integers(n_obstacles[0], n_obstacles[1] + 1))
        for _ in range(k):
            r = int(rng.integers(radius[0], radius[1] + 1))
            r = min(r, max(1, (ny - 4) // 2 - 1))
            cx = float(rng.uniform(0, nx))
            cy = float(rng.uniform(1 + r, ny - 2 - r)) if ny - 3 - 2 * r > 0 else ny / 2
            dx = np.minimum(np.abs(x - cx), nx - np.abs(x - cx))  # periodic in x
            m[(dx ** 2 + (y - cy) ** 2) <= r * r] = WALL
        H = ny - 2
        out.append({"nx": nx, "ny": ny, "mask": m, "force": (8.0 * nu * u_max / (H * H), 0.0)})
    return out
