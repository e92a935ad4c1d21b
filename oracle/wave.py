"""Oracle: Fourier Forwarding for the wave equation (Section 4.2, eqs. (4.7)-(4.12)).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

u_tt = c^2 (u_xx + u_yy) with u = f, u_t = g at t = 0 (eq. (4.7)).  One large step of
the interior propagator: the 2D-FC expansions F and G of the data (eq. (4.10)), the
modal solutions of eq. (4.11),
    a_lm(t) = hat f_lm cos(w t) + hat g_lm sin(w t)/w,   a_00(t) = hat f_00 + t hat g_00,
    w = 2 pi c sqrt((l/L_x)^2 + (m/L_y)^2),
and U_FC(., t) = sum a_lm(t) e^{2 pi i (l (x-a0)/L_x + m (y-b0)/L_y)} on the grid (inverse
DFT), together with its time derivative from a'_lm(t) = -w hat f sin(w t) + hat g cos(w t)
(needed as the initial velocity of the next large step, Section 4.2).  U_FC is the
solution at the grid points at distance >= c t from the curve (domain of dependence).

Reading: the paper prints the frequency as alpha_lm = (2 pi c)^2 [(l/L_x)^2 + (m/L_y)^2]
inside cos(alpha t); alpha is the square of the frequency w of the ODE
a'' + alpha a = 0 of eq. (4.11), so cos(w t) and sin(w t)/w with w = sqrt(alpha) are used.
"""
from __future__ import annotations

import numpy as np

from oracle import fc2d as F


def frequencies(grid, c):
    Lx, Ly = grid.nx * grid.h, grid.ny * grid.h
    l = np.arange(grid.nx // 2 + 1)
    m = np.fft.fftfreq(grid.ny, 1.0 / grid.ny)
    return 2 * np.pi * c * np.sqrt((l[None, :] / Lx) ** 2 + (m[:, None] / Ly) ** 2)


def advance_modes(Fh, Gh, w, t):
    """a(t) and a'(t) of eq. (4.12) (with w = sqrt(alpha))."""
    wz = np.where(w == 0, 1.0, w)
    a = Fh * np.cos(w * t) + Gh * np.where(w == 0, t, np.sin(w * t) / wz)
    at = -Fh * w * np.sin(w * t) + Gh * np.cos(w * t)
    return a, at


def interior_step(geo, mats, f_grid, f_bdry, g_grid, g_bdry, c, t, stencils=None):
    """U_FC(., t) and its time derivative on the whole grid (valid at distance >= c t)."""
    gr = geo.grid
    Fh = F.coefficients(F.extension(geo, mats, f_grid, f_bdry, stencils))
    Gh = F.coefficients(F.extension(geo, mats, g_grid, g_bdry, stencils))
    a, at = advance_modes(Fh, Gh, frequencies(gr, c), t)
    n = gr.nx * gr.ny
    u = np.fft.irfft2(a * n, s=(gr.ny, gr.nx))
    ut = np.fft.irfft2(at * n, s=(gr.ny, gr.nx))
    return u, ut
