"""Oracle: boundary, normals, Cartesian grid, inside test, feet of normals, strip set.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 3.1 (eqs. (3.2)-(3.7)), Section 3.3 and Section 3.4 of the paper.

Readings (the paper leaves these open):
* The boundary q(theta) is a trigonometric polynomial, oriented counter-clockwise
  (a clockwise input is re-parametrised by theta -> -theta).  The unit normal
  n = (y', -x')/|q'| then points out of the domain, as V+ in eq. (3.3) requires.
* Inside test (which grid points are in the closed domain): a grid point is inside
  when it lies in a closed interval [X_{2m}, X_{2m+1}] of the sorted crossings of
  its grid row with the curve (Jordan curve theorem / ray casting).  Crossings are
  the sign changes of the line's coordinate minus the curve's on 16 B uniform
  samples, refined; two consecutive crossings closer than 1e-7 times the grid box
  are a tangency artefact and are both dropped.
* The foot theta^Q of an exterior point Q is the parameter of the nearest point of
  the curve (the exact quantity the interpolant T(tau) of eq. (3.9) approximates),
  eta_Q = |Q - q(theta^Q)|.  The seed is the nearest of 16 B samples of the curve
  (a k-d tree); Newton's method on (q(theta) - Q).q'(theta) = 0 finishes it.
* H cap V+ (the strip set) is the set of grid points that are not inside and have
  0 < eta_Q <= C k1 (Section 3.1: V+ has 0 <= gamma <= C k1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial import cKDTree


# --------------------------------------------------------------------------- #
# The curve
# --------------------------------------------------------------------------- #
@dataclass
class Curve:
    cx: np.ndarray
    sx: np.ndarray
    cy: np.ndarray
    sy: np.ndarray

    @property
    def k(self):
        return np.arange(len(self.cx), dtype=np.float64)

    def _eval(self, a, b, theta, der):
        theta = np.asarray(theta, dtype=np.float64)
        out = np.zeros(theta.shape)
        for k in range(len(a)):
            if a[k] == 0.0 and b[k] == 0.0:
                continue
            c, s = np.cos(k * theta), np.sin(k * theta)
            if der == 0:
                out = out + a[k] * c + b[k] * s
            elif der == 1:
                out = out + k * (-a[k] * s + b[k] * c)
            elif der == 2:
                out = out - k * k * (a[k] * c + b[k] * s)
            else:
                out = out + k ** 3 * (a[k] * s - b[k] * c)
        return out

    def x(self, t, der=0):
        return self._eval(self.cx, self.sx, t, der)

    def y(self, t, der=0):
        return self._eval(self.cy, self.sy, t, der)

    def point(self, t):
        return self.x(t), self.y(t)

    def normal(self, t):
        """Outward unit normal (y', -x')/|q'| of a counter-clockwise curve."""
        xp, yp = self.x(t, 1), self.y(t, 1)
        s = np.hypot(xp, yp)
        return yp / s, -xp / s


def make_curve(boundary) -> Curve:
    """Curve of a ``workloads.Boundary``, re-parametrised to run counter-clockwise."""
    cx, sx, cy, sy = boundary.arrays()
    k = np.arange(len(cx))
    area = np.pi * np.sum(k * (cx * sy - sx * cy))
    if area < 0:
        sx, sy = -sx, -sy
    return Curve(cx.copy(), sx.copy(), cy.copy(), sy.copy())


# --------------------------------------------------------------------------- #
# Crossings of grid lines with the curve
# --------------------------------------------------------------------------- #
def _roots(f, fp, n_samples: int, samples=None):
    """All roots in [0, 2 pi) of the periodic function f, by sign changes on the
    uniform sample t_s = 2 pi s/n_s, s = 0..n_s, followed by bisection and two Newton
    steps.  ``samples`` may hold f(t_s) already."""
    th = 2 * np.pi * np.arange(n_samples + 1) / n_samples
    v = f(th) if samples is None else samples
    # the curve is closed: the sample at 2 pi is the one at 0 (f(2 pi) may round
    # differently and hide a root at theta = 0 between the two)
    v = np.append(v[:-1], v[0])
    pos = v > 0
    idx = np.nonzero(pos[:-1] != pos[1:])[0]
    if len(idx) == 0:
        return np.zeros(0)
    lo = th[idx].copy()
    hi = th[idx + 1].copy()
    flo = v[idx].copy()
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        same = (fm > 0) == (flo > 0)
        lo = np.where(same, mid, lo)
        flo = np.where(same, fm, flo)
        hi = np.where(same, hi, mid)
    r = 0.5 * (lo + hi)
    for _ in range(2):
        d = fp(r)
        step = np.where(d != 0, f(r) / np.where(d != 0, d, 1.0), 0.0)
        r = r - step
    return np.mod(r, 2 * np.pi)


def _drop_tangencies(X, tol):
    """Remove any two consecutive crossings closer than tol: a line that only touches
    the curve (a double root) can show up as such a pair when a sample lands exactly
    on the touching point; its position is then undetermined to ~1e-8."""
    out = []
    for x in X:
        if out and x - out[-1] < tol:
            out.pop()
        else:
            out.append(x)
    return np.array(out)


def crossings(curve: Curve, axis: str, value: float, n_samples: int, samples=None,
              tol: float = 0.0):
    """Sorted crossing coordinates of the curve with the line y = value (axis='row',
    returns x's) or x = value (axis='col', returns y's).  ``samples``: the curve
    coordinate (y for rows, x for columns) at the uniform sample points."""
    s = None if samples is None else samples - value
    if axis == "row":
        th = _roots(lambda t: curve.y(t) - value, lambda t: curve.y(t, 1), n_samples, s)
        return _drop_tangencies(np.sort(curve.x(th)), tol)
    th = _roots(lambda t: curve.x(t) - value, lambda t: curve.x(t, 1), n_samples, s)
    return _drop_tangencies(np.sort(curve.y(th)), tol)


@dataclass
class GridGeometry:
    """Everything the 2D-FC evaluation needs about one domain and grid."""
    curve: Curve
    grid: object
    params: object
    xs: np.ndarray                 # grid x coordinates
    ys: np.ndarray                 # grid y coordinates
    row_cross: list                # row j -> sorted crossing x's
    col_cross: list                # column i -> sorted crossing y's
    inside: np.ndarray             # bool [ny][nx]
    theta_p: np.ndarray            # boundary parameters theta_p = 2 pi p / B
    bx: np.ndarray                 # q(theta_p)
    by: np.ndarray
    nx_: np.ndarray                # n(theta_p)
    ny_: np.ndarray
    strip_lin: np.ndarray          # linear index j*nx + i of strip points (sorted)
    strip_theta: np.ndarray        # foot parameter theta^Q in [0, 2 pi)
    strip_eta: np.ndarray          # distance eta_Q
    bdry_x: np.ndarray             # all boundary points where f is needed:
    bdry_y: np.ndarray             #   B nodes, then column crossings, then row crossings
    col_offset: np.ndarray         # start of column i's crossings in the boundary list
    row_offset: np.ndarray         # start of row j's crossings in the boundary list


def n_crossing_samples(params) -> int:
    return 16 * params.B


def tangency_tolerance(grid) -> float:
    """Crossing pairs closer than 1e-7 times the larger side of the grid box are
    tangency artefacts (see _drop_tangencies)."""
    return 1e-7 * max(grid.nx, grid.ny) * grid.h


def build_geometry(w) -> GridGeometry:
    """Section 3.1 (boundary grid I_B, eq. (3.4); Cartesian grid H, eq. (3.7)),
    the inside test, and Sections 3.3-3.4 (feet of normals for H cap V+)."""
    curve = make_curve(w.boundary)
    g, p = w.grid, w.params
    xs = g.a0 + g.h * np.arange(g.nx)
    ys = g.b0 + g.h * np.arange(g.ny)
    ns = n_crossing_samples(p)
    ts = 2 * np.pi * np.arange(ns + 1) / ns
    sx, sy = curve.point(ts)
    tol = tangency_tolerance(g)
    row_cross = [crossings(curve, "row", y, ns, sy, tol) for y in ys]
    col_cross = [crossings(curve, "col", x, ns, sx, tol) for x in xs]
    inside = np.zeros((g.ny, g.nx), dtype=bool)
    for j, X in enumerate(row_cross):
        for m in range(0, len(X) - 1, 2):
            inside[j] |= (xs >= X[m]) & (xs <= X[m + 1])
    theta_p = 2 * np.pi * np.arange(p.B) / p.B
    bx, by = curve.point(theta_p)
    nxv, nyv = curve.normal(theta_p)
    # feet of the normals through exterior points near the curve
    n_dense = 16 * p.B
    td = 2 * np.pi * np.arange(n_dense) / n_dense
    tree = cKDTree(np.stack(curve.point(td), axis=1))
    X, Y = np.meshgrid(xs, ys)
    ext = ~inside
    cand = np.nonzero(ext.ravel())[0]
    qx, qy = X.ravel()[cand], Y.ravel()[cand]
    width = p.C * p.k1
    dist, nn = tree.query(np.stack([qx, qy], axis=1), distance_upper_bound=width + 2 * g.h)
    keep = np.isfinite(dist)
    cand, qx, qy, th = cand[keep], qx[keep], qy[keep], td[nn[keep]]
    th = newton_foot(curve, qx, qy, th)
    fx, fy = curve.point(th)
    eta = np.hypot(qx - fx, qy - fy)
    ok = (eta > 0) & (eta <= width)
    order = np.argsort(cand[ok], kind="stable")
    strip_lin = cand[ok][order]
    strip_theta = np.mod(th[ok][order], 2 * np.pi)
    strip_eta = eta[ok][order]
    # boundary data points: B nodes, column crossings, row crossings
    col_offset = np.zeros(g.nx + 1, dtype=np.int64)
    row_offset = np.zeros(g.ny + 1, dtype=np.int64)
    bdx, bdy = [bx], [by]
    off = p.B
    for i, Yc in enumerate(col_cross):
        col_offset[i] = off
        bdx.append(np.full(len(Yc), xs[i]))
        bdy.append(Yc)
        off += len(Yc)
    col_offset[g.nx] = off
    for j, Xc in enumerate(row_cross):
        row_offset[j] = off
        bdx.append(Xc)
        bdy.append(np.full(len(Xc), ys[j]))
        off += len(Xc)
    row_offset[g.ny] = off
    return GridGeometry(curve=curve, grid=g, params=p, xs=xs, ys=ys, row_cross=row_cross,
                        col_cross=col_cross, inside=inside, theta_p=theta_p, bx=bx, by=by,
                        nx_=nxv, ny_=nyv, strip_lin=strip_lin, strip_theta=strip_theta,
                        strip_eta=strip_eta, bdry_x=np.concatenate(bdx),
                        bdry_y=np.concatenate(bdy), col_offset=col_offset, row_offset=row_offset)


def newton_foot(curve: Curve, qx, qy, theta, iters: int = 40):
    """Newton's method on phi(theta) = (q(theta) - Q).q'(theta) = 0."""
    th = np.array(theta, dtype=np.float64)
    for _ in range(iters):
        x, y = curve.x(th), curve.y(th)
        xp, yp = curve.x(th, 1), curve.y(th, 1)
        xpp, ypp = curve.x(th, 2), curve.y(th, 2)
        phi = (x - qx) * xp + (y - qy) * yp
        dphi = xp * xp + yp * yp + (x - qx) * xpp + (y - qy) * ypp
        step = phi / dphi
        th = th - step
        if np.all(np.abs(step) < 1e-15):
            break
    return th
