"""Oracle: the 2D-FC Poisson solver (Section 4.1, eqs. (4.1)-(4.6)).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Delta u = f in the domain, u = g on the curve.  u = u_p + v (eq. (4.2)):

1. Particular solution (eqs. (4.5)-(4.6)).  hat f^c is the DFT of the 2D-FC extension
   of f.  b_{lm} = -hat f_{lm} / ((2 pi l/L_x)^2 + (2 pi m/L_y)^2), b_00 = 0, and
   u_p = hat f_00 (x^2 + y^2)/4 + sum b_{lm} e^{2 pi i (l (x-a0)/L_x + m (y-b0)/L_y)}
   on the grid (inverse DFT), with L_x = nx h, L_y = ny h.
   Reading: the paper's constant term carries a minus sign; with it Delta u_p would be
   f^c - 2 hat f_00, so the sign is taken as +, which gives Delta u_p = f^c exactly.
   The series is relative to the grid origin (phase convention of coefficients()).
2. u_p on the curve (Section 4.1): iterated 1D Lagrange interpolation of degree
   M_P - 1 (first along x on M_P grid rows, then along y), the M_P nodes of each
   direction centred on the point: i0 = floor((X - a0)/h) - (ceil(M_P/2) - 1).
3. Laplace problem for v with g_hom = g - u_p on the curve (eqs. (4.3)-(4.4)).  Reading
   of the "smooth-kernel integral equation with the Nystrom method": the interior
   Dirichlet problem as a double-layer potential
       v(x) = int phi(y) d/dnu(y) Phi(x, y) ds(y),  Phi = -(1/2 pi) ln|x - y|,
   whose interior limit gives the second-kind equation -phi/2 + K phi = g_hom.  The
   kernel is smooth on the curve (its diagonal limit is (x'' y' - x' y'')/(4 pi |q'|^2)),
   so the trapezoidal rule on N_b equispaced parameters converges super-algebraically.
   N_b = N_x (Section 4.1.1).  The dense system is solved directly (numpy.linalg.solve
   serves as the library primitive; the GPU uses GMRES).
4. v on the grid points inside: the trapezoidal sum.  Near-boundary reading of "local
   mesh refinement and interpolation of degree M_P - 1" (the paper refers the details
   to later work), with s = (2 pi / N_b) max |q'| (the largest node spacing) and R = 8:
   * points at distance >= 5 s use the N_b-point rule;
   * points at distance in [5 s/R, 5 s) use the rule on R N_b points, the density
     refined by trigonometric interpolation (zero-padded DFT);
   * points closer than 5 s/R take, along the normal through their foot, the degree
     M_P - 1 Lagrange interpolant through v on the curve (trigonometric interpolation of
     the nodal values g_hom) and the refined sums at distances 5s/R, ..., (M_P+3)s/R.
5. u = u_p + v at the grid points inside.

Parity of the near-boundary digits is unpinned by the paper (reading above); the
pins are the manufactured solutions, harmonic data and the paper's Table 3.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

from oracle import fc2d as F
from oracle import geometry as G


def particular(geo, mats, f_grid, f_bdry, stencils=None):
    """u_p on the whole grid H (eqs. (4.5)-(4.6), sign of the constant term as above)."""
    g = geo.grid
    ext = F.extension(geo, mats, f_grid, f_bdry, stencils)
    c = F.coefficients(ext)                        # [ny][nx/2+1], 1/(nx ny) normalised
    Lx, Ly = g.nx * g.h, g.ny * g.h
    l = np.arange(g.nx // 2 + 1)
    m = np.fft.fftfreq(g.ny, 1.0 / g.ny)
    den = (2 * np.pi * l[None, :] / Lx) ** 2 + (2 * np.pi * m[:, None] / Ly) ** 2
    den[0, 0] = 1.0
    b = -c / den
    b[0, 0] = 0.0
    up = np.fft.irfft2(b * (g.nx * g.ny), s=(g.ny, g.nx))
    X, Y = np.meshgrid(geo.xs, geo.ys)
    return up + c[0, 0].real * (X * X + Y * Y) / 4.0, c


def _window(coord0, h, n, x, MP):
    i0 = math.floor((x - coord0) / h) - ((MP + 1) // 2 - 1)
    i0 = min(max(i0, 0), n - MP)
    return np.arange(i0, i0 + MP)


def up_on_points(geo, up, X, Y, MP):
    """Iterated 1D interpolation of degree MP-1: along x on MP rows, then along y."""
    g = geo.grid
    out = np.zeros(len(X))
    for n, (x, y) in enumerate(zip(X, Y)):
        ii = _window(g.a0, g.h, g.nx, x, MP)
        jj = _window(g.b0, g.h, g.ny, y, MP)
        wx = F.lagrange_weights(geo.xs[ii], x)
        wy = F.lagrange_weights(geo.ys[jj], y)
        rows = np.array([np.dot(wx, up[j, ii]) for j in jj])
        out[n] = np.dot(wy, rows)
    return out


def bie_nodes(curve, Nb):
    t = 2 * np.pi * np.arange(Nb) / Nb
    x, y = curve.point(t)
    x1, y1 = curve.x(t, 1), curve.y(t, 1)
    x2, y2 = curve.x(t, 2), curve.y(t, 2)
    return t, x, y, x1, y1, x2, y2


def bie_matrix(curve, Nb):
    """Nystrom matrix of -phi/2 + K phi with the trapezoidal rule (weights 2 pi/Nb)."""
    t, x, y, x1, y1, x2, y2 = bie_nodes(curve, Nb)
    dx = x[:, None] - x[None, :]
    dy = y[:, None] - y[None, :]
    r2 = dx * dx + dy * dy
    np.fill_diagonal(r2, 1.0)
    k = (y1[None, :] * dx - x1[None, :] * dy) / (2 * np.pi * r2)
    diag = (x2 * y1 - x1 * y2) / (4 * np.pi * (x1 * x1 + y1 * y1))
    np.fill_diagonal(k, diag)
    return -0.5 * np.eye(Nb) + (2 * np.pi / Nb) * k


def double_layer(curve, Nb, phi, px, py):
    """v at points (px, py) by the trapezoidal sum (not for points on the curve)."""
    t, x, y, x1, y1, _, _ = bie_nodes(curve, Nb)
    out = np.zeros(len(px))
    for s in range(0, len(px), 4096):
        dx = px[s:s + 4096, None] - x[None, :]
        dy = py[s:s + 4096, None] - y[None, :]
        k = (y1[None, :] * dx - x1[None, :] * dy) / (2 * np.pi * (dx * dx + dy * dy))
        out[s:s + 4096] = (2 * np.pi / Nb) * (k @ phi)
    return out


def trig_interp(values, theta):
    """Trigonometric interpolant of equispaced periodic samples, at parameters theta."""
    Nb = len(values)
    c = np.fft.fft(values) / Nb
    k = np.fft.fftfreq(Nb, 1.0 / Nb)
    if Nb % 2 == 0:
        c[Nb // 2] *= 0.5
        c = np.append(c, c[Nb // 2])
        k = np.append(k, Nb // 2)
        k[Nb // 2] = -Nb // 2
    return np.real(np.exp(1j * np.outer(theta, k)) @ c)


def node_spacing(curve, Nb, n=4096):
    """Largest distance between neighbouring BIE nodes, (2 pi/Nb) max |q'(t)|."""
    t = 2 * np.pi * np.arange(n) / n
    return 2 * np.pi / Nb * np.max(np.hypot(curve.x(t, 1), curve.y(t, 1)))


def inside_feet(geo, width):
    """Feet and distances of the inside grid points closer than `width` to the curve."""
    g, p = geo.grid, geo.params
    curve = geo.curve
    n_dense = 16 * p.B
    td = 2 * np.pi * np.arange(n_dense) / n_dense
    tree = cKDTree(np.stack(curve.point(td), axis=1))
    X, Y = np.meshgrid(geo.xs, geo.ys)
    cand = np.nonzero(geo.inside.ravel())[0]
    qx, qy = X.ravel()[cand], Y.ravel()[cand]
    dist, nn = tree.query(np.stack([qx, qy], axis=1), distance_upper_bound=width + 2 * g.h)
    keep = np.isfinite(dist)
    cand, qx, qy, th = cand[keep], qx[keep], qy[keep], td[nn[keep]]
    th = G.newton_foot(curve, qx, qy, th)
    fx, fy = curve.point(th)
    eta = np.hypot(qx - fx, qy - fy)
    ok = eta < width
    return cand[ok], np.mod(th[ok], 2 * np.pi), eta[ok]


REFINE = 8


def refine_density(phi, R):
    """Trigonometric interpolation of the equispaced density to R times as many nodes."""
    Nb = len(phi)
    c = np.fft.fft(phi)
    big = np.zeros(R * Nb, complex)
    half = Nb // 2
    big[:half] = c[:half]
    big[-half:] = c[-half:]
    if Nb % 2 == 0:
        big[half] = 0.5 * c[half]
        big[-half] = 0.5 * c[half]
    else:
        big[half] = c[half]
    return np.real(np.fft.ifft(big)) * R


def laplace_on_grid(geo, phi, ghom, Nb, MP, R=REFINE):
    """v at every inside grid point (step 4)."""
    curve = geo.curve
    s = node_spacing(curve, Nb)
    delta = 5.0 * s
    X, Y = np.meshgrid(geo.xs, geo.ys)
    lin_in = np.nonzero(geo.inside.ravel())[0]
    v = np.zeros(geo.inside.size)
    near_lin, near_th, near_eta = inside_feet(geo, delta)
    far = np.setdiff1d(lin_in, near_lin, assume_unique=True)
    v[far] = double_layer(curve, Nb, phi, X.ravel()[far], Y.ravel()[far])
    if len(near_lin):
        phiR = refine_density(phi, R)
        mid = near_eta >= delta / R
        ml = near_lin[mid]
        v[ml] = double_layer(curve, R * Nb, phiR, X.ravel()[ml], Y.ravel()[ml])
        cl, cth, ceta = near_lin[~mid], near_th[~mid], near_eta[~mid]
        if len(cl):
            nx_, ny_ = curve.normal(cth)
            fx, fy = curve.point(cth)
            nodes = np.concatenate([[0.0], (delta + s * np.arange(MP - 1)) / R])
            vals = np.zeros((len(cl), MP))
            vals[:, 0] = trig_interp(ghom, cth)
            for j in range(1, MP):
                vals[:, j] = double_layer(curve, R * Nb, phiR, fx - nodes[j] * nx_,
                                          fy - nodes[j] * ny_)
            for n in range(len(cl)):
                w = F.lagrange_weights(nodes, ceta[n])
                v[cl[n]] = np.dot(w, vals[n])
    return v.reshape(geo.inside.shape)


def solve(geo, mats, f_grid, f_bdry, g_nodes, Nb=None, MP=None, stencils=None):
    """u = u_p + v at the inside grid points (0 elsewhere), plus intermediates."""
    g, p = geo.grid, geo.params
    Nb = Nb or g.nx
    MP = MP or p.M
    up, c = particular(geo, mats, f_grid, f_bdry, stencils)
    t, bx, by, *_ = bie_nodes(geo.curve, Nb)
    upb = up_on_points(geo, up, bx, by, MP)
    ghom = g_nodes - upb
    phi = np.linalg.solve(bie_matrix(geo.curve, Nb), ghom)
    v = laplace_on_grid(geo, phi, ghom, Nb, MP)
    u = np.where(geo.inside, up + v, 0.0)
    return {"u": u, "up": up, "upb": upb, "phi": phi, "v": v, "coef": c}


def bie_points(curve, Nb):
    """The BIE nodes q(2 pi k/Nb), where the Dirichlet data g is needed."""
    _, x, y, *_ = bie_nodes(curve, Nb)
    return x, y
