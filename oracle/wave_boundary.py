"""Oracle: the Fourier Forwarding near-boundary solver U_B (Section 4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper only sketches U_B: an explicit small-step scheme on a set Omega_B that
contains the part of the domain within c Delta T of the curve, second-order Taylor
time stepping at CFL 0.125 (Section 4.2.1), Dirichlet data imposed "as in
Appelo-Petersson 2012" (SIAM J. Sci. Comput. 34: an embedded boundary, ghost values
beyond the curve from an interpolating polynomial through the boundary datum and
interior values along each grid line), and values at the inner edge of Omega_B taken
from the interior propagator U_FC.  Reading (the steps below are the definition the
library follows; every constant is named here):

* Band.  delta = n_c h.  The unknowns of U_B are the grid points of H cap Omega at a
  distance < delta + 2h from the curve (the distance to the nearest curve point, its
  foot found by Newton's method as for the strip points).  "Interface" points are the
  other grid points of H cap Omega that the formulas below reference; they are at a
  distance >= delta + 2h > c (Delta T + Delta t) from the curve, where U_FC is the
  solution (domain of dependence), and take U_FC's values.
* Chords.  A grid line meets H cap Omega in chords: the runs of inside points between
  two consecutive crossings X_a < X_b of the line with the curve (the plan's boundary
  points).  For a point P of a chord, k- and k+ count the chord points before and after
  it.
* Slaved points (the small-cell treatment).  A chord end point closer than XI_MIN h to
  its crossing (along x or y) is not stepped: its value is the boundary polynomial of
  that side (below) evaluated at the point, at every time level.  When a point could be
  slaved from several sides, the closest crossing wins (ties: x before y, lower side
  first).
* Decisions on a threshold carry a margin TIE = 2^-30 (in units of h): a point is in
  the band if dist < delta + 2h - TIE h, U_B's solution point if dist < delta - TIE h,
  slaved if xi < XI_MIN - TIE, and a later side replaces an earlier one only if its xi
  is smaller by more than TIE.  Symmetric grids put points exactly on these thresholds
  (the unit disk on a grid through the origin with h = 1/16 has points at distance
  exactly 6h), where two correct evaluations of the distance or the crossing differ in
  the last bit; the margin makes every implementation decide such points alike.
* Boundary polynomial of a chord side.  The degree <= Q_DEG Lagrange interpolant through
  the crossing of that side (the Dirichlet datum) and the Q_DEG non-slaved chord points
  nearest to it; on a chord with fewer non-slaved points it takes all of them and the
  other crossing's datum.
* Second differences.  u_xx + u_yy at an unknown P: along each axis the central
  difference of order 2 hw with half-width hw = min(R_FD, k- + 1, k+ + 1) (so at most
  one value beyond each crossing is used); a neighbour inside the chord takes its value
  (unknown, slaved or interface), the one neighbour beyond a crossing its "ghost" value:
  the boundary polynomial of that side at the ghost's coordinate.
* Dissipation.  B holds the fourth differences (1, -4, 6, -4, 1)/16 over every window
  of DISS_P + 1 = 5 consecutive non-slaved points of a chord that holds an unknown;
  D = B^T B / 2 (symmetric, positive semi-definite, norm <= 1).
* Time stepping (second-order Taylor, Section 4.2.1): Delta t = Delta T/(8 n_c), i.e.
  c Delta t = h/8 (CFL 0.125),
      u^1     = u^0 + Delta t u_t^0 + (c Delta t)^2/2 L(u^0),
      u^{n+1} = 2 u^n - u^{n-1} + (c Delta t)^2 L(u^n) - SIGMA D(u^n - u^{n-1}),
  L the second differences above with the Dirichlet data and interface values at t_n,
  D acting on the unknowns' and interface values' increments.  Without the
  dissipation term the semi-discrete operator of any such closure has eigenvalues off
  the real axis (a growth of 1e-3 per small step on the unit disk); SIGMA = 0.3 brings
  the spectral radius of the one-step map below 1 on every grid tested.

The combination with U_FC (eq. (4.9)) and the large steps are in ``oracle/wave.py``.
Parity unpinned by the paper: the digits of U_B follow this reading; the pins are the
plane wave of Section 4.2.1's first example and the Dirichlet eigenmodes of the disk
(exact solutions), the spectral radius of the one-step map, and polynomial exactness
of the difference formulas.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

from oracle import geometry as G

R_FD = 4        # half-width of the interior central difference (order 8)
Q_DEG = 3       # degree of the boundary polynomial
XI_MIN = 0.5    # chord end points closer than XI_MIN h to their crossing are slaved
DISS_P = 4      # order of the differences in the dissipation
SIGMA = 0.3     # dissipation coefficient
BAND_EXTRA = 2  # the band reaches delta + BAND_EXTRA h from the curve
CFL = 0.125     # c Delta t / h
TIE = 2.0 ** -30  # decision margin (below)


def central_weights(hw: int) -> np.ndarray:
    """Weights (times 1/h^2) of the order-2hw central second difference on the offsets
    -hw..hw, in closed form: w_k = 2 (-1)^(k+1) (hw!)^2 / (k^2 (hw-k)! (hw+k)!) for
    k != 0 and w_0 = -2 sum_{k=1}^{hw} 1/k^2 (the unique symmetric stencil exact for
    polynomials of degree <= 2hw + 1)."""
    from math import factorial
    w = np.zeros(2 * hw + 1)
    for k in range(1, hw + 1):
        v = 2.0 * (-1) ** (k + 1) * factorial(hw) ** 2 / (k * k * factorial(hw - k) * factorial(hw + k))
        w[hw + k] = w[hw - k] = v
    w[hw] = -2.0 * sum(1.0 / (k * k) for k in range(1, hw + 1))
    return w


def lagrange(nodes, x) -> np.ndarray:
    nodes = np.asarray(nodes, dtype=np.float64)
    w = np.ones(len(nodes))
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            if k != j:
                w[j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return w


def inside_distance(geo, dmax: float) -> np.ndarray:
    """Distance to the curve of the inside grid points within ~dmax of it (inf for the
    others): nearest of 64 B curve samples, then Newton's method on the foot equation
    (q(theta) - P).q'(theta) = 0, as for the strip points (Section 3.4)."""
    curve, g = geo.curve, geo.grid
    n_dense = 64 * geo.params.B
    td = 2 * np.pi * np.arange(n_dense) / n_dense
    tree = cKDTree(np.stack(curve.point(td), axis=1))
    X, Y = np.meshgrid(geo.xs, geo.ys)
    cand = np.nonzero(geo.inside.ravel())[0]
    qx, qy = X.ravel()[cand], Y.ravel()[cand]
    d0, nn = tree.query(np.stack([qx, qy], axis=1), distance_upper_bound=dmax + 4 * g.h)
    keep = np.isfinite(d0)
    th = G.newton_foot(curve, qx[keep], qy[keep], td[nn[keep]])
    fx, fy = curve.point(th)
    out = np.full(X.size, np.inf)
    out[cand[keep]] = np.hypot(qx[keep] - fx, qy[keep] - fy)
    return out.reshape(X.shape)


@dataclass
class Band:
    """U_B's unknowns, slaved points, interface points and operators.

    Operators act on (u at the unknowns, values at the interface points, Dirichlet
    data at the plan's boundary points): each is a dict of sparse matrices 'u', 'f',
    'g' with one row per unknown (L, B) or per slaved point (S)."""
    n_c: int
    delta: float
    reach: float                     # the band's outer distance from the curve
    dist: np.ndarray                 # [ny][nx] distance of inside points (inf: far)
    unknown_lin: np.ndarray          # linear indices of the unknowns
    slaved_lin: np.ndarray           # linear indices of the slaved points
    iface_lin: np.ndarray            # linear indices of the interface points
    L: dict = field(default_factory=dict)
    Bd: dict = field(default_factory=dict)
    S: dict = field(default_factory=dict)


class _Builder:
    def __init__(self, geo, n_c, reach_cells=None):
        self.geo = geo
        g = geo.grid
        self.h, self.nx, self.ny = g.h, g.nx, g.ny
        self.ins = geo.inside
        self.delta = n_c * g.h
        reach = (n_c + BAND_EXTRA if reach_cells is None else reach_cells) * g.h
        self.reach = reach
        self.dist = inside_distance(geo, reach)
        self.band = self.ins & (self.dist < reach - TIE * g.h)
        # slaving
        self.slave = {}
        for j, i in zip(*np.nonzero(self.band)):
            best = None
            for axis in (0, 1):
                for side in (-1, 1):
                    if self._inside(j, i, axis, side):
                        continue
                    cr = self._crossing(j, i, axis, side)
                    if cr is None:  # the point lies on the curve where this line touches it
                        continue
                    xi = abs(cr[0] - self._coord(j, i, axis)) / self.h
                    if xi < XI_MIN - TIE and (best is None or xi < best[0] - TIE):
                        best = (xi, axis, side)
            if best is not None:
                self.slave[(j, i)] = best[1:]
        self.unknown = self.band.copy()
        for (j, i) in self.slave:
            self.unknown[j, i] = False
        self.uidx = -np.ones(self.ins.shape, dtype=np.int64)
        lin_u = np.nonzero(self.unknown.ravel())[0]
        self.uidx.ravel()[lin_u] = np.arange(len(lin_u))
        self.lin_u = lin_u
        self.iface = {}

    # grid-line helpers (axis 0: along x in row j; axis 1: along y in column i)
    def _step(self, j, i, axis, k):
        return (j, i + k) if axis == 0 else (j + k, i)

    def _coord(self, j, i, axis):
        return self.geo.xs[i] if axis == 0 else self.geo.ys[j]

    def _inside(self, j, i, axis, k):
        jj, ii = self._step(j, i, axis, k)
        return bool(self.ins[jj, ii])

    def _crossing(self, j, i, axis, side):
        """(coordinate, plan boundary index) of the crossing bounding the chord of
        (j, i) on `side` (-1: lower coordinate, +1: upper).  The chord is the closed
        inside interval [X_2k, X_2k+1] of the sorted crossings that holds the point."""
        geo = self.geo
        c = self._coord(j, i, axis)
        if axis == 0:
            X, off = geo.row_cross[j], geo.row_offset[j]
        else:
            X, off = geo.col_cross[i], geo.col_offset[i]
        m = int(np.searchsorted(X, c, side="right")) - 1  # last crossing <= c
        lo = m - (m % 2)
        if lo < 0 or lo + 1 >= len(X) or not (X[lo] <= c <= X[lo + 1]):
            return None  # no chord of this line holds the point (a tangency)
        m = lo + (1 if side > 0 else 0)
        return float(X[m]), int(off + m)

    def _count(self, j, i, axis, side):
        k = 0
        while self._inside(j, i, axis, (k + 1) * side):
            k += 1
        return k

    def key(self, j, i):
        """Key of the value at an inside grid point: unknown, slaved (expanded by the
        caller) or interface."""
        if self.unknown[j, i]:
            return ("u", int(self.uidx[j, i]))
        lin = j * self.nx + i
        if lin not in self.iface:
            self.iface[lin] = len(self.iface)
        return ("f", self.iface[lin])

    def poly(self, j, i, axis, side, x):
        """Boundary polynomial of the chord side of (j, i), at coordinate x (a form)."""
        cr = self._crossing(j, i, axis, side)
        if cr is None:
            raise ValueError(f"grid point ({j}, {i}) has no chord along axis {axis}")
        X, b = cr
        k = self._count(j, i, axis, side)
        jj, ii = self._step(j, i, axis, k * side)  # chord end point on that side
        nodes, keys = [X], [("g", b)]
        while len(nodes) < Q_DEG + 1:
            if not self.ins[jj, ii]:
                X2, b2 = self._crossing(j, i, axis, -side)
                nodes.append(X2)
                keys.append(("g", b2))
                break
            if (jj, ii) not in self.slave:
                nodes.append(self._coord(jj, ii, axis))
                keys.append(self.key(jj, ii))
            jj, ii = self._step(jj, ii, axis, -side)
        form = {}
        for w, kk in zip(lagrange(nodes, x), keys):
            form[kk] = form.get(kk, 0.0) + w
        return form

    def value(self, j, i):
        if (j, i) in self.slave:
            axis, side = self.slave[(j, i)]
            return self.poly(j, i, axis, side, self._coord(j, i, axis))
        return {self.key(j, i): 1.0}

    def laplacian_row(self, j, i):
        form = {}
        h2 = self.h * self.h
        for axis in (0, 1):
            km = self._count(j, i, axis, -1)
            kp = self._count(j, i, axis, +1)
            hw = min(R_FD, km + 1, kp + 1)
            w = central_weights(hw)
            for k in range(-hw, hw + 1):
                if k < -km or k > kp:  # beyond the crossing: ghost value
                    side = 1 if k > 0 else -1
                    jj, ii = self._step(j, i, axis, k)
                    f2 = self.poly(j, i, axis, side, self._coord(jj, ii, axis))
                else:
                    f2 = self.value(*self._step(j, i, axis, k))
                for kk, v in f2.items():
                    form[kk] = form.get(kk, 0.0) + w[k + hw] * v / h2
        return form

    def dissipation_rows(self):
        from math import comb
        p = DISS_P
        coef = np.array([(-1) ** (p - k) * comb(p, k) for k in range(p + 1)], float) / 2.0 ** p
        rows = []
        ok = self.ins.copy()
        for (j, i) in self.slave:
            ok[j, i] = False
        for axis in (0, 1):
            for lin in self.lin_u:
                j, i = divmod(int(lin), self.nx)
                for start in range(-p, 1):
                    pts = [self._step(j, i, axis, start + k) for k in range(p + 1)]
                    if not all(ok[a, b] for a, b in pts):
                        continue
                    # each window once: counted at its first unknown
                    first = next(q for q in pts if self.unknown[q])
                    if first != (j, i):
                        continue
                    form = {}
                    for cw, q in zip(coef, pts):
                        kk = self.key(*q)
                        form[kk] = form.get(kk, 0.0) + cw
                    rows.append(form)
        return rows


def _assemble(rows, n_u, n_f, n_g):
    out = {}
    for kind, ncol in (("u", n_u), ("f", n_f), ("g", n_g)):
        r_, c_, v_ = [], [], []
        for ri, form in enumerate(rows):
            for (k, c), v in form.items():
                if k == kind:
                    r_.append(ri)
                    c_.append(c)
                    v_.append(v)
        out[kind] = sp.csr_matrix((np.array(v_, float), (np.array(r_, int), np.array(c_, int))),
                                  shape=(len(rows), ncol))
    return out


def build_band(geo, n_c: int, reach_cells=None) -> Band:
    """The near-boundary solver's sets and operators for large-step width delta = n_c h;
    the band reaches reach_cells h from the curve (default n_c + 2; the small-square
    interface procedure needs a deeper band, ``oracle/wave_squares.py``)."""
    b = _Builder(geo, n_c, reach_cells)
    lap = [b.laplacian_row(*divmod(int(lin), b.nx)) for lin in b.lin_u]
    dis = b.dissipation_rows()
    slaved = sorted(j * b.nx + i for (j, i) in b.slave)
    srows = [b.value(*divmod(lin, b.nx)) for lin in slaved]
    n_u, n_f, n_g = len(b.lin_u), len(b.iface), int(len(geo.bdry_x))
    iface_lin = np.zeros(n_f, dtype=np.int64)
    for lin, k in b.iface.items():
        iface_lin[k] = lin
    band = Band(n_c=n_c, delta=b.delta, reach=b.reach, dist=b.dist,
                unknown_lin=b.lin_u.astype(np.int64),
                slaved_lin=np.array(slaved, dtype=np.int64), iface_lin=iface_lin)
    band.L = _assemble(lap, n_u, n_f, n_g)
    band.Bd = _assemble(dis, n_u, n_f, n_g)
    band.S = _assemble(srows, n_u, n_f, n_g)
    return band


def laplacian(band: Band, u, f, g):
    """L(u) at the unknowns: second differences with interface values f and Dirichlet
    data g."""
    return band.L["u"] @ u + band.L["f"] @ f + band.L["g"] @ g


def dissipation(band: Band, du, df):
    """D applied to the increments (du at the unknowns, df at the interface points)."""
    return band.Bd["u"].T @ (band.Bd["u"] @ du + band.Bd["f"] @ df) / 2


def slaved_values(band: Band, u, f, g):
    return band.S["u"] @ u + band.S["f"] @ f + band.S["g"] @ g


def first_step(band: Band, h, u0, ut0, f0, g0, dt):
    """u^1 = u^0 + dt u_t^0 + (c dt)^2/2 L(u^0) with c dt = CFL h."""
    cdt = CFL * h
    return u0 + dt * ut0 + 0.5 * cdt * cdt * laplacian(band, u0, f0, g0)


def step(band: Band, h, u, u_prev, f, f_prev, g):
    """u^{n+1} = 2u^n - u^{n-1} + (c dt)^2 L(u^n) - SIGMA D(u^n - u^{n-1})."""
    cdt = CFL * h
    return (2 * u - u_prev + cdt * cdt * laplacian(band, u, f, g)
            - SIGMA * dissipation(band, u - u_prev, f - f_prev))


def one_step_matrix(band: Band, h, sigma: float = SIGMA) -> np.ndarray:
    """The one-small-step map (u^n, u^{n-1}) -> (u^{n+1}, u^n) with homogeneous data,
    as a dense matrix (for the stability pin); sigma: the dissipation coefficient."""
    cdt = CFL * h
    A = band.L["u"].toarray()
    Bu = band.Bd["u"].toarray()
    D = Bu.T @ Bu / 2
    N = A.shape[0]
    I = np.eye(N)
    return np.block([[2 * I + cdt * cdt * A - sigma * D, -I + sigma * D],
                     [I, np.zeros((N, N))]])
