"""Plain, slow, FP64 CPU oracle for the lattice Boltzmann hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it.  It shares no code, table or helper with
the CUDA library; the two meet only through seeded inputs from
``paper_2311_16080_gb300.inputs`` (which holds no LBM arithmetic).

Everything here is written as the paper states it, array-at-a-time with numpy,
without blocking, fusion or reordering:

* collision then streaming, Eqs. 1-2 (Section 2);
* BGK relaxation, Eq. 3, with omega = dt/tau and tau from Eq. 4;
* the quadratic equilibrium of Eq. 5, used by every collision model;
* density and velocity moments, Eqs. 6-7;
* periodic streaming as a toroidal shift per direction (``np.roll``), which is
  how Section 3.4 describes streaming;
* boundary conditions driven by a per-cell type mask (Section 3.5);
* the exact-difference body force (Section 6.1, the corrector force equation);
* the KBC entropic collision named in Section 2 (formula from Karlin, Bosch and
  Chikatamarla 2014, which the paper cites; the paper prints none);
* a hand-derived reverse-mode adjoint of the step (Section 3.6 takes gradients
  of ``step``; Section 7 lists adjoint-based optimisation as future work).

Array convention: populations are ``f[i, z, y, x]`` in 3D and ``f[i, y, x]`` in
2D (x fastest, like the GPU's SoA layout); velocities are ``u[a, ...]`` with
a = x, y, z.  All functions accept real or complex arrays so that complex-step
derivatives can pin the adjoint.

Readings of points the paper leaves open:

* weights w_i are not printed (Section 2 only names them); the standard
  D2Q9 / D3Q19 / D3Q27 weights are used, pinned by the lattice isotropy
  identities in the tests;
* velocity order follows Figure 1 with the rest velocity first;
* one step is f_{t+1} = S_bc(C(f_t)): collision on fluid-like cells, then a
  pull stream in which the mask decides what replaces a population whose source
  cell is not fluid (Section 3.5 / 3.6 allow BCs after collision or after
  streaming; here every rule is folded into the pull);
* halfway bounce-back for WALL (stationary) and LID (moving, with the
  momentum term 2 w_i rho_w (c_i . u_w) / c_s^2 and rho_w fixed);
* EQ cells hold f^eq(rho_w, u_w) (the equilibrium BC of Section 3.5 / 5);
* INLET cells are velocity boundaries (inward normal +x unless set): Zou-He
  reconstruction of the populations entering the fluid (non-equilibrium
  bounce-back of every unknown, no transverse term), or the regularized rule;
* OUTLET cells copy their c_x = -1 populations from the cell at x-1
  (zero-gradient extrapolation);
* observables are those of the post-stream state f_t; the reported velocity
  with a body force is (j + F/2) / rho;
* solid (WALL, LID) cells report rho = 0, u = 0;
* FWALL cells are full-way bounce-back walls (the walls of the paper's
  performance setup, Section 5): they are streamed like any cell, their
  collision reverses every population (f*_i = f_opp(i)), they start at rest
  and report rho = 0, u = 0.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Cell types of the per-cell mask (Section 3.5).  The numeric codes are the
# library's public ABI values; the oracle keeps its own copy.
FLUID, WALL, LID, INLET, OUTLET, EQ, FWALL = 0, 1, 2, 3, 4, 5, 6
FLUID_LIKE = (FLUID, INLET, OUTLET)

CS2 = 1.0 / 3.0  # speed of sound squared, Section 2 (after Eq. 4)


# ---------------------------------------------------------------------------
# Lattices (Figure 1; Section 3.2)

_FIG1 = {
    9: [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)],
    19: [(1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0), (0, -1, 0), (0, 0, -1),
         (1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0), (1, 0, 1), (1, 0, -1),
         (-1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1)],
}
_FIG1[27] = _FIG1[19] + [(1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1),
                         (-1, 1, 1), (-1, 1, -1), (-1, -1, 1), (-1, -1, -1)]

# Weight by |c|^2 (standard values; the paper does not print them).
_WEIGHTS = {
    9: {0: Fraction(4, 9), 1: Fraction(1, 9), 2: Fraction(1, 36)},
    19: {0: Fraction(1, 3), 1: Fraction(1, 18), 2: Fraction(1, 36)},
    27: {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)},
}


class Lattice:
    """Velocity set c_i, weights w_i and opposite index opp(i) of one lattice."""

    def __init__(self, q: int):
        if q not in _FIG1:
            raise ValueError(f"unknown lattice Q={q}")
        d = 2 if q == 9 else 3
        vel = [tuple([0] * d)] + list(_FIG1[q])
        self.q = q
        self.d = d
        self.c = np.array(vel, dtype=np.int64)                     # (Q, d)
        self.w_frac = [_WEIGHTS[q][sum(v * v for v in ci)] for ci in vel]
        self.w = np.array([float(x) for x in self.w_frac])         # (Q,)
        self.opp = np.array([vel.index(tuple(-v for v in ci)) for ci in vel])

    # spatial axes of a population plane f[i] are (z, y, x) or (y, x)
    def _axes(self):
        return tuple(range(self.d))

    def _shift(self, i):
        """Roll amounts, in array-axis order, that move a value at x to x + c_i."""
        ci = self.c[i]
        return tuple(int(v) for v in ci[::-1])  # (cz, cy, cx) or (cy, cx)

    def roll(self, a, i, sign=1):
        """Return b with b(x) = a(x - sign * c_i), periodic in every axis."""
        return np.roll(a, tuple(sign * s for s in self._shift(i)), axis=self._axes())


# ---------------------------------------------------------------------------
# Moments and equilibrium (Eqs. 5-7)

def density(lat: Lattice, f):
    """rho = sum_i f_i (Eq. 6)."""
    return f.sum(axis=0)


def momentum(lat: Lattice, f):
    """j = sum_i c_i f_i, so that u = j / rho (Eq. 7)."""
    return np.stack([np.tensordot(lat.c[:, a].astype(float), f, axes=(0, 0))
                     for a in range(lat.d)])


def equilibrium(lat: Lattice, rho, u):
    """Quadratic equilibrium of Eq. 5:
    f_i^eq = w_i rho [1 + c_i.u / cs2 + (c_i.u)^2 / (2 cs2^2) - |u|^2 / (2 cs2)].
    """
    usq = sum(u[a] * u[a] for a in range(lat.d))
    out = []
    for i in range(lat.q):
        cu = sum(lat.c[i, a] * u[a] for a in range(lat.d))
        out.append(lat.w[i] * rho * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2)
                                     - usq / (2 * CS2)))
    return np.stack(out)


# ---------------------------------------------------------------------------
# Collision operators (Eq. 3; KBC of Karlin et al. 2014)

def omega_from_nu(nu):
    """omega = dt / tau with tau = nu / cs2 + dt / 2 (Eq. 4), dt = 1."""
    return 1.0 / (nu / CS2 + 0.5)


def nu_from_omega(omega):
    """Inverse of Eq. 4 with dt = 1."""
    return CS2 * (1.0 / omega - 0.5)


def collide_bgk(lat: Lattice, f, omega):
    """BGK, Eq. 3: f* = f - omega (f - f^eq(rho, u))."""
    rho = density(lat, f)
    u = momentum(lat, f) / rho
    return f - omega * (f - equilibrium(lat, rho, u))


# One-dimensional inverse of the natural moments {sum f, sum c f, sum c^2 f}
# on the three velocities {-1, 0, +1}: f(c) = M0 a0(c) + M1 a1(c) + M2 a2(c).
def _a0(c):
    return 1.0 if c == 0 else 0.0


def _a1(c):
    return 0.5 * c if c != 0 else 0.0


def _a2(c):
    return -1.0 if c == 0 else 0.5


def kbc_shear_part(lat: Lattice, g):
    """Shear part s(g) of a population field g in the KBC decomposition.

    s carries exactly the deviatoric second moments of g (the off-diagonal
    Pi_ab and the traceless normal parts Pi_aa - tr(Pi)/d) and no other
    natural moment; it is built with the product-lattice inverse of the
    natural moments (Karlin, Bosch, Chikatamarla 2014; Bosch et al. 2015).
    Defined on the tensor-product lattices D2Q9 and D3Q27 only.
    """
    if lat.q not in (9, 27):
        raise ValueError("KBC shear part is defined on D2Q9 and D3Q27 only")
    d = lat.d
    cf = lat.c.astype(float)
    Pi = [[np.tensordot(cf[:, a] * cf[:, b], g, axes=(0, 0)) for b in range(d)]
          for a in range(d)]
    tr = sum(Pi[a][a] for a in range(d))
    out = []
    for i in range(lat.q):
        ci = lat.c[i]
        s = 0.0 * g[0]
        for a in range(d):                       # traceless normal stresses
            coef = _a2(ci[a])
            for b in range(d):
                if b != a:
                    coef *= _a0(ci[b])
            if coef != 0.0:
                s = s + coef * (Pi[a][a] - tr / d)
        for a in range(d):                       # off-diagonal stresses
            for b in range(a + 1, d):
                coef = _a1(ci[a]) * _a1(ci[b])
                for e in range(d):
                    if e != a and e != b:
                        coef *= _a0(ci[e])
                if coef != 0.0:
                    s = s + coef * Pi[a][b]
        out.append(s)
    return np.stack(out)


def kbc_gamma(lat: Lattice, ds, dh, feq, beta, tiny=1e-30):
    """Entropic stabiliser gamma = 1/beta - (2 - 1/beta) <ds|dh> / <dh|dh>,
    <a|b> = sum_i a_i b_i / f_i^eq.  Where <dh|dh> < tiny, gamma = 2 (BGK)."""
    sh = (ds * dh / feq).sum(axis=0)
    hh = (dh * dh / feq).sum(axis=0)
    safe = np.where(np.abs(hh) < tiny, 1.0, hh)
    g = 1.0 / beta - (2.0 - 1.0 / beta) * sh / safe
    return np.where(np.abs(hh) < tiny, 2.0, g)


def collide_kbc(lat: Lattice, f, omega, gamma=None):
    """KBC entropic multi-relaxation collision (Section 2 names it).

    f = k + s + h; ds = s(f - f^eq), dh = (f - f^eq) - ds;
    beta = omega / 2; f* = f - beta (2 ds + gamma dh).
    ``gamma`` overrides the entropic value (gamma = 2 reduces to BGK).
    """
    rho = density(lat, f)
    u = momentum(lat, f) / rho
    feq = equilibrium(lat, rho, u)
    fneq = f - feq
    ds = kbc_shear_part(lat, fneq)
    dh = fneq - ds
    beta = 0.5 * omega
    g = kbc_gamma(lat, ds, dh, feq, beta) if gamma is None else gamma
    return f - beta * (2.0 * ds + g * dh)


def force_increment(lat: Lattice, f, F):
    """Exact-difference body force (Kupershtokh 2004, as used in Section 6.1):
    f^eq(rho, u + F/rho) - f^eq(rho, u) with u = j / rho and dt = 1."""
    rho = density(lat, f)
    u = momentum(lat, f) / rho
    du = np.stack([F[a] / rho for a in range(lat.d)])
    return equilibrium(lat, rho, u + du) - equilibrium(lat, rho, u)


# ---------------------------------------------------------------------------
# Boundary description and the step

class BC:
    """Prescribed values of the mask's boundary types.

    lid_u / lid_rho:  moving-wall velocity and fixed wall density (LID cells).
    inlet_u:          Zou-He inlet velocity (INLET cells): d constants, or a
                      field of shape (d, *mask.shape) (a velocity profile).
    eq_rho / eq_u:    equilibrium-BC state (EQ cells).
    wall_q:           Bouzidi wall distances: None, or an array (Q, *mask.shape)
                      whose entry [i, x] is the fraction q in [0, 1] of the
                      link from fluid cell x along c_i at which the wall
                      crosses it, where x + c_i is a WALL cell; NaN elsewhere
                      (those links keep halfway bounce-back, q = 1/2).
    inlet_scheme:     "zou_he" or "regularized", the two inflow rules Section
                      4.3 names for INLET cells.
    inlet_normal:     (axis, sign): the direction n = sign e_axis from the
                      INLET cells' boundary into the fluid; (0, +1), inflow
                      along +x, by default.  INLET cells are velocity
                      boundaries: with the velocity parallel to the wall they
                      are a moving wall (the regularized lid of Section 4.2).
    """

    def __init__(self, d, lid_u=None, lid_rho=1.0, inlet_u=None, eq_rho=1.0, eq_u=None, wall_q=None,
                 inlet_scheme="zou_he", inlet_normal=(0, 1)):
        z = [0.0] * d
        self.lid_u = list(lid_u) if lid_u is not None else z
        self.lid_rho = lid_rho
        if inlet_u is None:
            self.inlet_u = z
        elif np.ndim(inlet_u) > 1:
            self.inlet_u = np.asarray(inlet_u, dtype=float)
        else:
            self.inlet_u = list(inlet_u)
        self.eq_rho = eq_rho
        self.eq_u = list(eq_u) if eq_u is not None else z
        self.wall_q = wall_q
        self.inlet_scheme = inlet_scheme  # "zou_he" | "regularized"
        self.inlet_normal = (int(inlet_normal[0]), int(inlet_normal[1]))


def _const_feq(lat, rho, u):
    return equilibrium(lat, np.array(rho, dtype=float),
                       np.array(u, dtype=float).reshape(lat.d))


def fluid_like(mask):
    return np.isin(mask, FLUID_LIKE)


def bouzidi(lat: Lattice, h, mask, j, q):
    """Linear interpolated bounce-back of Bouzidi, Firdaouss and Lallemand
    (2001), the curved-wall no-slip rule Section 4.3 names: the population
    f_j(x) that a fluid cell x pulls from a WALL cell x - c_j, when the wall
    crosses the link from x along c_i = -c_j at the fraction q of its length:
      q <  1/2:  f_j(x) = 2q h_i(x) + (1 - 2q) h_i(x + c_j)
      q >= 1/2:  f_j(x) = h_i(x) / (2q) + (2q - 1) / (2q) h_j(x)
    (h: post-collision populations).  Where q < 1/2 but x + c_j is not a
    FLUID cell the halfway value h_i(x) is kept.  Returns the field of f_j
    values for every x (meaningful where q is finite)."""
    i = lat.opp[j]
    behind = lat.roll(h[i], i)               # h_i(x - c_i) = h_i(x + c_j)
    behind_fl = lat.roll(mask, i) == FLUID
    with np.errstate(invalid="ignore", divide="ignore"):
        low = np.where(behind_fl, 2.0 * q * h[i] + (1.0 - 2.0 * q) * behind, h[i])
        high = h[i] / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * h[j]
    return np.where(q < 0.5, low, high)


def pull_plain(lat: Lattice, h, mask, bc: BC):
    """Post-stream populations from post-collision ones, before the inlet and
    outlet rules: f_i(x) = h_i(x - c_i) with periodic wrap (Eq. 2), except that
    a source cell x - c_i of type WALL gives h_opp(i)(x) (or the Bouzidi value
    where bc.wall_q gives the link a wall distance), LID gives
    h_opp(i)(x) + 2 w_i rho_w (c_i . u_w) / cs2, and EQ gives f_i^eq(rho_w, u_w)."""
    feq_w = _const_feq(lat, bc.eq_rho, bc.eq_u)
    out = []
    for i in range(lat.q):
        g = lat.roll(h[i], i)
        src = lat.roll(mask, i)
        hb = h[lat.opp[i]]
        cu_lid = sum(lat.c[i, a] * bc.lid_u[a] for a in range(lat.d))
        if bc.wall_q is not None and i != 0:
            q = bc.wall_q[lat.opp[i]]
            hb = np.where(np.isfinite(q), bouzidi(lat, h, mask, i, q), hb)
        g = np.where(src == WALL, hb, g)
        g = np.where(src == LID, hb + 2.0 * lat.w[i] * bc.lid_rho * cu_lid / CS2, g)
        g = np.where(src == EQ, feq_w[i], g)
        out.append(g)
    return np.stack(out)


def _inlet_setup(lat: Lattice, mask, bc: BC):
    """Velocity boundary at INLET cells with inward normal n = sign e_axis:
    c.n of every direction, the prescribed velocity field and the density
    from the known populations (those with c.n <= 0),
      rho = [sum_{c.n=0} f_i + 2 sum_{c.n=-1} f_i] / (1 - u.n)."""
    axis, sign = bc.inlet_normal
    cn = sign * lat.c[:, axis]
    uin = np.stack([np.broadcast_to(np.asarray(bc.inlet_u[a], dtype=float), mask.shape)
                    for a in range(lat.d)])
    return cn, uin, sign * uin[axis]


def zou_he_inlet(lat: Lattice, f, mask, bc: BC):
    """Zou-He velocity boundary on INLET cells: the unknown populations are
    those entering the fluid through the boundary (c_i . n = +1; with the
    default normal, the inflow along +x, c_x = +1):
      rho = [sum_{c.n=0} f_i + 2 sum_{c.n=-1} f_i] / (1 - u.n),
      f_i = f_opp(i) + f_i^eq(rho, u) - f_opp(i)^eq(rho, u) for each unknown i."""
    sel = mask == INLET
    if not sel.any():
        return f
    f = f.copy()
    cn, uin, un = _inlet_setup(lat, mask, bc)
    rho = (sum(f[i] for i in range(lat.q) if cn[i] == 0)
           + 2.0 * sum(f[i] for i in range(lat.q) if cn[i] == -1)) / (1.0 - un)
    feq = equilibrium(lat, rho, uin)
    for i in range(lat.q):
        if cn[i] == 1:
            j = lat.opp[i]
            f[i] = np.where(sel, f[j] + feq[i] - feq[j], f[i])
    return f


def regularized_inlet(lat: Lattice, f, mask, bc: BC):
    """Regularized velocity boundary of Latt et al. (2008), the second inflow
    rule Section 4.3 names (and, as a moving wall, the regularized lid of
    Section 4.2), on INLET cells (unknowns c_i . n = +1):
      rho as in the Zou-He rule; f^neq_i = f_i - f_i^eq(rho, u) for the known
      populations and f^neq_i = f^neq_opp(i) for the unknown ones;
      Pi = sum_i c_i c_i f^neq_i; then every population is replaced by
      f_i = f_i^eq(rho, u) + w_i / (2 cs^4) (c_i c_i - cs^2 I) : Pi."""
    sel = mask == INLET
    if not sel.any():
        return f
    cn, uin, un = _inlet_setup(lat, mask, bc)
    rho = (sum(f[i] for i in range(lat.q) if cn[i] == 0)
           + 2.0 * sum(f[i] for i in range(lat.q) if cn[i] == -1)) / (1.0 - un)
    feq = equilibrium(lat, rho, uin)
    neq = f - feq
    for i in range(lat.q):
        if cn[i] == 1:
            neq[i] = neq[lat.opp[i]]
    Pi = [[sum(lat.c[i, a] * lat.c[i, b] * neq[i] for i in range(lat.q)) for b in range(lat.d)]
          for a in range(lat.d)]
    out = f.copy()
    for i in range(lat.q):
        qpi = sum((lat.c[i, a] * lat.c[i, b] - (CS2 if a == b else 0.0)) * Pi[a][b]
                  for a in range(lat.d) for b in range(lat.d))
        out[i] = np.where(sel, feq[i] + lat.w[i] / (2.0 * CS2 * CS2) * qpi, f[i])
    return out


def outflow(lat: Lattice, f_plain, f, mask):
    """Zero-gradient outflow on OUTLET cells (Section 4.3 cites an
    extrapolation outflow): populations with c_x = -1 take the value that the
    pull rule gives at the cell x - 1.  The unknown populations entering at
    the outlet are thereby the outlet plane's own post-collision c_x = -1
    populations, moved transversally, so the mass lost per step equals the
    plane's x-momentum, and a flow uniform in x passes unchanged."""
    sel = mask == OUTLET
    if not sel.any():
        return f
    f = f.copy()
    for i in range(lat.q):
        if lat.c[i, 0] == -1:
            left = np.roll(f_plain[i], 1, axis=lat.d - 1)  # value at x - 1
            f[i] = np.where(sel, left, f[i])
    return f


def stream_bc(lat: Lattice, h, mask, bc: BC):
    """S_bc: the pull stream with every boundary rule of the mask applied."""
    fp = pull_plain(lat, h, mask, bc)
    f = (regularized_inlet if bc.inlet_scheme == "regularized" else zou_he_inlet)(lat, fp, mask, bc)
    f = outflow(lat, fp, f, mask)
    # non-fluid cells carry fixed values: EQ cells f^eq(rho_w, u_w), solids a
    # rest state that no rule ever reads.
    feq_w = _const_feq(lat, bc.eq_rho, bc.eq_u)
    solid = (mask == WALL) | (mask == LID)
    for i in range(lat.q):
        f[i] = np.where(mask == EQ, feq_w[i], f[i])
        f[i] = np.where(solid, lat.w[i], f[i])
    return f


class Params:
    """Collision model and parameters of one run."""

    def __init__(self, lat, omega, collision="bgk", force=None, bc=None, kbc_gamma=None):
        self.omega = omega
        self.collision = collision  # "bgk" | "kbc" | "none"
        self.force = list(force) if force is not None else None
        self.bc = bc if bc is not None else BC(lat.d)
        self.kbc_gamma = kbc_gamma


def collide(lat: Lattice, f, mask, p: Params):
    """C: collision (+ body force) on fluid-like cells; FWALL cells reverse
    their populations (full-way bounce-back); identity elsewhere."""
    if p.collision == "none":
        return f
    if p.collision == "bgk":
        h = collide_bgk(lat, f, p.omega)
    elif p.collision == "kbc":
        h = collide_kbc(lat, f, p.omega, gamma=p.kbc_gamma)
    else:
        raise ValueError(p.collision)
    if p.force is not None:
        h = h + force_increment(lat, f, p.force)
    fl = fluid_like(mask)
    out = np.where(fl[None], h, f)
    fw = mask == FWALL
    if fw.any():
        out = np.where(fw[None], f[lat.opp], out)
    return out


def step(lat: Lattice, f, mask, p: Params):
    """One time step f_{t+1} = S_bc(C(f_t)) (Eqs. 1-2 with Section 3.5 BCs)."""
    return stream_bc(lat, collide(lat, f, mask, p), mask, p.bc)


def run(lat: Lattice, f, mask, p: Params, n: int):
    for _ in range(n):
        f = step(lat, f, mask, p)
    return f


def init_state(lat: Lattice, rho, u, mask, p: Params):
    """f_0 = f^eq(rho, u) on fluid-like cells (Eq. 5); boundary cells take the
    fixed values of the mask types."""
    f = equilibrium(lat, rho, u)
    feq_w = _const_feq(lat, p.bc.eq_rho, p.bc.eq_u)
    solid = (mask == WALL) | (mask == LID) | (mask == FWALL)
    for i in range(lat.q):
        f[i] = np.where(mask == EQ, feq_w[i], f[i])
        f[i] = np.where(solid, lat.w[i], f[i])
    return f


def macroscopic(lat: Lattice, f, mask, p: Params):
    """Reported rho and u of a post-stream state (Eqs. 6-7).  Fluid-like cells
    report u = (j + F/2) / rho under a body force; solids report zeros."""
    rho = density(lat, f)
    j = momentum(lat, f)
    if p.force is not None:
        fl = fluid_like(mask)
        j = np.stack([j[a] + np.where(fl, 0.5 * p.force[a], 0.0) for a in range(lat.d)])
    u = j / rho
    solid = (mask == WALL) | (mask == LID) | (mask == FWALL)
    rho = np.where(solid, 0.0, rho)
    u = np.where(solid[None], 0.0, u)
    return rho, u


# ---------------------------------------------------------------------------
# Reverse mode (hand-derived adjoint of the step)

def equilibrium_vjp(lat: Lattice, rho, j, gbar):
    """Given gbar = dL/df^eq, return (dL/drho, dL/dj) of f^eq written in
    (rho, j): f_i^eq = w_i [rho + 3 c_i.j + 4.5 (c_i.j)^2 / rho - 1.5 |j|^2 / rho]
    (Eq. 5 with u = j / rho and cs2 = 1/3)."""
    u = j / rho
    usq = sum(u[a] * u[a] for a in range(lat.d))
    rbar = 0.0 * rho
    jbar = [0.0 * rho for _ in range(lat.d)]
    for i in range(lat.q):
        cu = sum(lat.c[i, a] * u[a] for a in range(lat.d))
        rbar = rbar + gbar[i] * lat.w[i] * (1.0 - 4.5 * cu * cu + 1.5 * usq)
        for a in range(lat.d):
            jbar[a] = jbar[a] + gbar[i] * lat.w[i] * (3.0 * lat.c[i, a] + 9.0 * cu * lat.c[i, a]
                                                       - 3.0 * u[a])
    return rbar, np.stack(jbar)


def _moments_vjp(lat, rbar, jbar):
    """Adjoint of (rho, j) = (sum_i f_i, sum_i c_i f_i)."""
    return np.stack([rbar + sum(lat.c[k, a] * jbar[a] for a in range(lat.d))
                     for k in range(lat.q)])


def collide_bgk_vjp(lat: Lattice, f, omega, hbar, force=None):
    """VJP of h = (1 - omega) f + omega f^eq(rho, j) [+ f^eq(rho, j + F) - f^eq(rho, j)]."""
    rho = density(lat, f)
    j = momentum(lat, f)
    if force is None:
        rb, jb = equilibrium_vjp(lat, rho, j, omega * hbar)
    else:
        rb1, jb1 = equilibrium_vjp(lat, rho, j, (omega - 1.0) * hbar)
        jF = np.stack([j[a] + force[a] for a in range(lat.d)])
        rb2, jb2 = equilibrium_vjp(lat, rho, jF, hbar)
        rb, jb = rb1 + rb2, jb1 + jb2
    return (1.0 - omega) * hbar + _moments_vjp(lat, rb, jb)


def stream_bc_vjp(lat: Lattice, fbar, mask, bc: BC):
    """Transpose of the linear part of S_bc on fluid-like cells (periodic,
    WALL, LID, EQ; the inlet and outlet rules have no adjoint here).
    A population f_i(x) at a fluid-like cell x depends on h_i(x - c_i) when the
    source is fluid-like, on h_opp(i)(x) for a WALL or LID source, and on no
    h for an EQ source."""
    if np.isin(mask, (INLET, OUTLET, FWALL)).any():
        raise ValueError("adjoint of the inlet/outlet and full-way rules is not defined")
    fl = fluid_like(mask)
    hbar = np.zeros_like(fbar)
    for i in range(lat.q):
        g = np.where(fl, fbar[i], 0.0)
        src = lat.roll(mask, i)
        src_fl = fluid_like(src)
        # h_i(y) feeds f_i(y + c_i): shift g back by c_i
        hbar[i] = hbar[i] + lat.roll(np.where(src_fl, g, 0.0), i, sign=-1)
        bb = (src == WALL) | (src == LID)
        hbar[lat.opp[i]] = hbar[lat.opp[i]] + np.where(bb, g, 0.0)
    return hbar


def collide_vjp(lat: Lattice, f, mask, p: Params, hbar):
    if p.collision == "none":
        return hbar
    if p.collision != "bgk":
        raise ValueError("adjoint is defined for BGK only")
    fb = collide_bgk_vjp(lat, f, p.omega, hbar, p.force)
    fl = fluid_like(mask)
    return np.where(fl[None], fb, hbar)


def macroscopic_seed(lat: Lattice, f, mask, p: Params, rbar, ubar):
    """dL/df of a loss given through the cotangents (rbar, ubar) of the
    reported observables rho = sum f, u = (j + F/2) / rho:
    fbar_i = rbar + ubar . (c_i - u) / rho on fluid-like cells, 0 elsewhere."""
    rho, u = macroscopic(lat, f, mask, p)
    fl = fluid_like(mask)
    safe = np.where(fl, rho, 1.0)
    out = []
    for i in range(lat.q):
        v = rbar + sum(ubar[a] * (lat.c[i, a] - u[a]) for a in range(lat.d)) / safe
        out.append(np.where(fl, v, 0.0))
    return np.stack(out)


def kinetic_energy(lat: Lattice, f, mask, p: Params, box):
    """L = sum over the box of (1/2) rho |u|^2 of the reported observables
    (complex-safe: no absolute values)."""
    rho, u = macroscopic(lat, f, mask, p)
    ke = 0.5 * rho * sum(u[a] * u[a] for a in range(lat.d))
    return ke[box].sum()


def kinetic_energy_grads(rho, u, box):
    """(dL/drho, dL/du) of ``kinetic_energy``: (1/2)|u|^2 and rho u on the box."""
    inb = np.zeros(rho.shape, dtype=bool)
    inb[box] = True
    rbar = np.where(inb, 0.5 * sum(u[a] * u[a] for a in range(u.shape[0])), 0.0)
    ubar = np.stack([np.where(inb, rho * u[a], 0.0) for a in range(u.shape[0])])
    return rbar, ubar


def gradient_init(lat: Lattice, rho0, u0, mask, p: Params, n, seed_fn):
    """Reverse-mode gradient of L(f_n) with respect to the initial fields of
    f_0 = f^eq(rho0, u0): stores every f_t, then runs the adjoint backwards.
    ``seed_fn(rho_n, u_n) -> (dL/drho, dL/du)`` gives the loss cotangents of
    the reported observables of f_n.
    Returns (dL/drho0, dL/du0) on fluid-like cells."""
    fs = [init_state(lat, rho0, u0, mask, p)]
    for _ in range(n):
        fs.append(step(lat, fs[-1], mask, p))
    rho_n, u_n = macroscopic(lat, fs[-1], mask, p)
    rb, ub = seed_fn(rho_n, u_n)
    fbar = macroscopic_seed(lat, fs[-1], mask, p, rb, ub)
    for t in range(n - 1, -1, -1):
        hbar = stream_bc_vjp(lat, fbar, mask, p.bc)
        fbar = collide_vjp(lat, fs[t], mask, p, hbar)
    fl = fluid_like(mask)
    fbar = np.where(fl[None], fbar, 0.0)
    j0 = np.stack([rho0 * u0[a] for a in range(lat.d)])
    rb0, jb0 = equilibrium_vjp(lat, rho0, j0, fbar)
    # chain (rho, j) -> (rho, u): j = rho u
    drho = rb0 + sum(jb0[a] * u0[a] for a in range(lat.d))
    du = np.stack([jb0[a] * rho0 for a in range(lat.d)])
    return drho, du


# ---------------------------------------------------------------------------
# Reductions used by the invariant checks

def wall_force(lat: Lattice, f, mask, p: Params, solid=None):
    """Momentum-exchange force on the WALL cells (Mei et al. 2002, in the
    form Caiazzo and Junk 2008 give for interpolated walls, the method Section
    4.3 names) in the update that starts from the post-stream state f: with
    h = C(f) and f' = S_bc(h) the next post-stream state,
      F = sum over links (x, i), x FLUID, x + c_i a WALL cell in `solid`
          (all WALL cells if None), of c_i [h_i(x) + f'_opp(i)(x)],
    the momentum the populations crossing each link hand to the wall."""
    h = collide(lat, f, mask, p)
    fn = stream_bc(lat, h, mask, p.bc)
    sel = (mask == WALL) if solid is None else ((mask == WALL) & solid)
    F = np.zeros(lat.d)
    for i in range(1, lat.q):
        tgt = lat.roll(sel.astype(np.uint8), i, sign=-1).astype(bool)   # x + c_i selected
        link = (mask == FLUID) & tgt
        v = np.where(link, h[i] + fn[lat.opp[i]], 0.0)
        for a in range(lat.d):
            F[a] += lat.c[i, a] * float(np.real(v.sum()))
    return F


def total_mass(lat: Lattice, f, mask):
    return float(np.real(density(lat, f)[fluid_like(mask)].sum()))


def total_momentum(lat: Lattice, f, mask):
    j = momentum(lat, f)
    fl = fluid_like(mask)
    return [float(np.real(j[a][fl].sum())) for a in range(lat.d)]
