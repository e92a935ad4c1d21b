"""Oracle: Fourier Forwarding for the wave equation (Section 4.2, eqs. (4.7)-(4.12)).

forward_wave (below) is the whole method: U_FC on the interior combined with the
near-boundary solver U_B of ``oracle/wave_boundary.py`` by eq. (4.9), large step after
large step.

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


def forward_wave(geo, mats, band, c, n_large, u0, ut0, g_fun=None, gt_fun=None,
                 stencils=None, squares=None, mats_1d=None):
    """The Fourier Forwarding solution (eq. (4.9)) after n_large large steps.

    Large step Delta T = n_c h / c (delta = c Delta T = n_c h, Section 4.2).  For each
    large step j (T_j = j Delta T):
      1. F, G: the 2D-FC expansions (eq. (4.10)) of u(T_j) and u_t(T_j) on H cap Omega
         with the Dirichlet data g(T_j) and its time derivative on the curve;
      2. U_FC(T_j + s Delta t) (eqs. (4.8), (4.12)) at the interface points of U_B, by a
         full inverse DFT at each small step s = 0..S, S = 8 n_c (the paper's faster
         small-square procedure is not followed here);
      3. S small steps of U_B (``oracle/wave_boundary.py``); U_B is continued across
         large steps (the first small step of all uses the Taylor start);
      4. u(T_{j+1}) = U_FC(T_{j+1}) where dist >= delta, U_B(T_{j+1}) where dist < delta
         (with the decision margin of ``oracle/wave_boundary.py``)
         (eq. (4.9)); u_t(T_{j+1}) = dU_FC/dt there, and at the U_B points the central
         difference (u^{N+1} - u^{N-1})/(2 Delta t) with u^{N+1} one further small step
         taken with this large step's U_FC (valid at the interface points for
         s = S + 1, since they lie farther than delta + h/8 from the curve); at slaved
         points the boundary polynomial of the time derivatives.
    g_fun(t), gt_fun(t): Dirichlet data and its time derivative at the plan's boundary
    points (None: zero).  u0, ut0: [ny][nx] (values outside the domain are ignored).
    stencils: the matching stencils of the geometry (computed when None).
    squares: a placement of ``oracle/wave_squares.py`` (with a band built for it): the
    interface values of the small steps then come from the small squares' expansions
    (the paper's small-square procedure) instead of the full inverse DFT; mats_1d: the
    d = 4 FC matrices of the squares' 1D continuations (default: mats).
    Returns u, u_t on [ny][nx] (zero outside the domain)."""
    from oracle import wave_boundary as WB
    gr = geo.grid
    h, ny, nx = gr.h, gr.ny, gr.nx
    S = 8 * band.n_c
    dT = band.n_c * h / c
    dt = dT / S
    zero_b = np.zeros(len(geo.bdry_x))
    gval = g_fun if g_fun is not None else (lambda t: zero_b)
    gtval = gt_fun if gt_fun is not None else (lambda t: zero_b)
    w = frequencies(gr, c)
    n = nx * ny
    inside = geo.inside
    near = inside & (band.dist < band.delta - WB.TIE * h)
    u = np.where(inside, u0, 0.0)
    ut = np.where(inside, ut0, 0.0)
    uu = u.ravel()[band.unknown_lin]
    u_prev = f_prev = None
    st = stencils if stencils is not None else F.matching_stencils(geo)
    for j in range(n_large):
        T = j * dT
        Fh = F.coefficients(F.extension(geo, mats, u, gval(T), st))
        Gh = F.coefficients(F.extension(geo, mats, ut, gtval(T), st))

        def ufc(tau, deriv=False):
            a, at = advance_modes(Fh, Gh, w, tau)
            return np.fft.irfft2((at if deriv else a) * n, s=(ny, nx))

        if squares is not None:
            from oracle import wave_squares as WS
            sq_spec = WS.square_spectra(geo, mats_1d if mats_1d is not None else mats,
                                        squares, u, ut)
        for s in range(S):
            m = j * S + s
            if squares is None:
                f = ufc(s * dt).ravel()[band.iface_lin]
            else:
                f = WS.evaluate(geo, squares, sq_spec, band.iface_lin, h, c, s * dt)
            g = gval(m * dt)
            if m == 0:
                un = WB.first_step(band, h, uu, ut.ravel()[band.unknown_lin], f, g, dt)
            else:
                un = WB.step(band, h, uu, u_prev, f, f_prev, g)
            u_prev, uu, f_prev = uu, un, f
        T1 = (j + 1) * dT
        Ug, Utg = ufc(dT), ufc(dT, True)
        fN, ftN = Ug.ravel()[band.iface_lin], Utg.ravel()[band.iface_lin]
        gN, gtN = gval(T1), gtval(T1)
        u_extra = WB.step(band, h, uu, u_prev, fN, f_prev, gN)
        ut_u = (u_extra - u_prev) / (2 * dt)
        u_new, ut_new = Ug.ravel().copy(), Utg.ravel().copy()
        nr = near.ravel()
        sel = nr[band.unknown_lin]
        u_new[band.unknown_lin[sel]] = uu[sel]
        ut_new[band.unknown_lin[sel]] = ut_u[sel]
        if len(band.slaved_lin):
            us = WB.slaved_values(band, uu, fN, gN)
            uts = WB.slaved_values(band, ut_u, ftN, gtN)
            sel = nr[band.slaved_lin]
            u_new[band.slaved_lin[sel]] = us[sel]
            ut_new[band.slaved_lin[sel]] = uts[sel]
        u = np.where(inside, u_new.reshape(ny, nx), 0.0)
        ut = np.where(inside, ut_new.reshape(ny, nx), 0.0)
    return u, ut
