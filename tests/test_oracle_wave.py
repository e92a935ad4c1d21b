"""Pins for the oracle Fourier Forwarding interior propagator (Section 4.2)."""
import numpy as np

import workloads as W
from oracle import fc2d as F
from oracle import geometry as G
from oracle import wave as V
from oracle.fc_matrices import load_fc_matrices
from tests.fc2d_check import paper_setup


def test_modal_advance_is_exact_for_box_modes():
    """A single Fourier mode of the periodic box travels exactly: a(t) = f cos(wt) + g
    sin(wt)/w reproduces cos(k.x - w t) for f = cos(k.x), g = w sin(k.x)."""
    g = W.workload("disk64").grid
    x, y = g.coords()
    X, Y = np.meshgrid(x - g.a0, y - g.b0)
    Lx, Ly = g.nx * g.h, g.ny * g.h
    kx, ky = 2 * np.pi * 3 / Lx, 2 * np.pi * -5 / Ly
    c = 1.3
    w = c * np.hypot(kx, ky)
    f = np.cos(kx * X + ky * Y)
    gg = w * np.sin(kx * X + ky * Y)
    Fh, Gh = np.fft.rfft2(f) / f.size, np.fft.rfft2(gg) / f.size
    t = 0.37
    a, at = V.advance_modes(Fh, Gh, V.frequencies(g, c), t)
    u = np.fft.irfft2(a * f.size, s=f.shape)
    ut = np.fft.irfft2(at * f.size, s=f.shape)
    assert np.abs(u - np.cos(kx * X + ky * Y - w * t)).max() < 1e-13
    assert np.abs(ut - w * np.sin(kx * X + ky * Y - w * t)).max() < 1e-12


def test_zero_time_returns_the_extension_and_constant_mode_grows_linearly():
    Fh = np.array([[2.0 + 0j, 1.0]])
    Gh = np.array([[0.5 + 0j, 0.0]])
    w = np.array([[0.0, 3.0]])
    a, at = V.advance_modes(Fh, Gh, w, 0.0)
    assert np.allclose(a, Fh) and np.allclose(at, Gh)
    a, at = V.advance_modes(Fh, Gh, w, 2.0)
    assert np.isclose(a[0, 0], 2.0 + 2.0 * 0.5) and np.isclose(at[0, 0], 0.5)


def test_plane_wave_inside_the_domain_of_dependence():
    """Example 4.3's plane waves u = cos(2k(x+t)/3) + cos(k(y+t)) on the unit disk: after
    one large step T the propagated 2D-FC expansion matches the exact solution at the
    grid points farther than c T from the curve, to the extension's accuracy."""
    k = 4 * np.pi
    u = lambda x, y, t: np.cos(2 * k * (x + t) / 3) + np.cos(k * (y + t))
    ut = lambda x, y, t: -(2 * k / 3) * np.sin(2 * k * (x + t) / 3) - k * np.sin(k * (y + t))
    mats = load_fc_matrices()
    w = paper_setup(W.disk(), 0.01)
    geo = G.build_geometry(w)
    st = F.matching_stencils(geo)
    T = 0.08
    f0, g0 = (lambda x, y: u(x, y, 0.0)), (lambda x, y: ut(x, y, 0.0))
    U, Ut = V.interior_step(geo, mats, W.grid_values(w, f0), F.boundary_values(geo, f0),
                            W.grid_values(w, g0), F.boundary_values(geo, g0), 1.0, T, st)
    X, Y = np.meshgrid(geo.xs, geo.ys)
    valid = geo.inside & (1.0 - np.hypot(X, Y) >= T)
    err = np.abs(U - u(X, Y, T))[valid].max()
    errt = np.abs(Ut - ut(X, Y, T))[valid].max()
    assert err < 1e-5 and errt < 1e-3 * k, (err, errt)
    # outside the domain of dependence the free-space propagation is not the solution
    bad = geo.inside & (1.0 - np.hypot(X, Y) < 0.2 * T)
    assert np.abs(U - u(X, Y, T))[bad].max() > 10 * err
