"""Pins for the oracle near-boundary solver U_B and the whole Fourier Forwarding solve
(Section 4.2): difference weights and closure exact for polynomials, the dissipation
symmetric positive semi-definite, the one-small-step map stable (spectral radius <= 1)
where the undamped closure is not, and the FF solution converging to two exact
solutions: the plane waves of Section 4.2.1's first example and a Dirichlet eigenmode
of the unit disk."""
import numpy as np
import pytest
from scipy.special import jn_zeros, jv

import workloads as W
from oracle import geometry as G
from oracle import wave as V
from oracle import wave_boundary as WB
from oracle.fc_matrices import load_fc_matrices
from tests.fc2d_check import paper_setup


def _disk(h, offset=(0.0, 0.0)):
    w = paper_setup(W.disk(), h, d=4)
    g = w.grid
    if offset != (0.0, 0.0):
        g = W.Grid(a0=g.a0 - offset[0] * h, b0=g.b0 - offset[1] * h, h=h, nx=g.nx, ny=g.ny)
        w = W.Workload(w.name, w.boundary, g, w.params)
    return w, G.build_geometry(w)


def test_central_weights_are_exact_to_their_order():
    """The closed-form order-2hw weights differentiate x^k exactly for k <= 2hw + 1 and
    miss x^(2hw+2) (the order is not higher)."""
    for hw in range(1, 5):
        w = WB.central_weights(hw)
        k = np.arange(-hw, hw + 1, dtype=float)
        for p in range(2 * hw + 2):
            exact = 2.0 if p == 2 else 0.0
            assert abs(w @ k ** p - exact) < 1e-11, (hw, p)
        assert abs(w @ k ** (2 * hw + 2)) > 1e-3


@pytest.mark.parametrize("name,h", [("disk", 0.05), ("disk", 0.043), ("kite", 0.0366)])
def test_closure_reproduces_cubics(name, h):
    """With exact Dirichlet data and interface values, the second differences with their
    ghost values equal the Laplacian of every cubic at every unknown, and the slaved
    values equal the cubic (the boundary polynomial has degree 3, the stencils order
    >= 2).  A wrong ghost index, sign or node set fails this."""
    if name == "disk":
        w, geo = _disk(h, (0.31, 0.17))
    else:
        w = W.workload("kite160x144")
        geo = G.build_geometry(w)
    band = WB.build_band(geo, 6)
    X, Y = np.meshgrid(geo.xs, geo.ys)
    cases = [(lambda x, y: 1 + 2 * x - 3 * y, lambda x, y: 0 * x),
             (lambda x, y: 1 + x ** 3 - 2 * x * x * y + 0.5 * y ** 3 + x * y,
              lambda x, y: 6 * x - 4 * y + 3 * y)]
    for u, lap in cases:
        U = u(X, Y).ravel()
        g = u(geo.bdry_x, geo.bdry_y)
        Lu = WB.laplacian(band, U[band.unknown_lin], U[band.iface_lin], g)
        scale = 1.0 / h ** 2
        assert np.abs(Lu - lap(X, Y).ravel()[band.unknown_lin]).max() < 1e-12 * scale * 100
        sv = WB.slaved_values(band, U[band.unknown_lin], U[band.iface_lin], g)
        assert np.abs(sv - U[band.slaved_lin]).max() < 1e-12
    # the sets: unknowns and slaved points are the band (inside, distance < delta + 2h),
    # interface points are inside and farther
    inside = geo.inside.ravel()
    d = band.dist.ravel()
    reach = band.delta + WB.BAND_EXTRA * h - WB.TIE * h
    assert inside[band.unknown_lin].all() and (d[band.unknown_lin] < reach).all()
    assert inside[band.iface_lin].all() and (d[band.iface_lin] >= reach).all()
    assert len(set(band.unknown_lin) | set(band.slaved_lin)) == int((inside & (d < reach)).sum())


def test_dissipation_is_symmetric_positive_semidefinite():
    w, geo = _disk(0.05, (0.31, 0.17))
    band = WB.build_band(geo, 6)
    Bu = band.Bd["u"].toarray()
    ev = np.linalg.eigvalsh(Bu.T @ Bu / 2)
    assert ev.min() > -1e-13 and ev.max() <= 1.0 + 1e-12


@pytest.mark.parametrize("h,offset", [(0.04, (0.0, 0.0)), (0.0403, (0.31, 0.17)),
                                      (0.0337, (0.31, 0.17)), (0.029, (0.12, 0.57))])
def test_one_small_step_map_is_stable(h, offset):
    """Spectral radius of (u^n, u^{n-1}) -> (u^{n+1}, u^n) (homogeneous data) on the unit
    disk, n_c = 8: <= 1 + 1e-12 with the dissipation."""
    w, geo = _disk(h, offset)
    band = WB.build_band(geo, 8)
    rad = np.abs(np.linalg.eigvals(WB.one_step_matrix(band, h))).max()
    assert rad <= 1 + 1e-12, rad


def test_the_closure_without_dissipation_grows():
    """Without the dissipation the closure alone is not stable in 2D (its eigenvalues
    leave the real axis): the one-step map's radius exceeds 1 + 1e-4 (unit disk,
    h = 0.04)."""
    w, geo = _disk(0.04)
    band = WB.build_band(geo, 8)
    rad0 = np.abs(np.linalg.eigvals(WB.one_step_matrix(band, 0.04, sigma=0.0))).max()
    assert rad0 > 1 + 1e-4, rad0


def test_one_small_step_map_is_stable_on_the_kite():
    geo = G.build_geometry(W.workload("kite160x144"))
    band = WB.build_band(geo, 6)
    h = geo.grid.h
    assert np.abs(np.linalg.eigvals(WB.one_step_matrix(band, h))).max() <= 1 + 1e-12


def _plane_wave(kap):
    u = lambda x, y, t: np.cos(2 * kap * (x + t) / 3) + np.cos(kap * (y + t))
    ut = lambda x, y, t: (-(2 * kap / 3) * np.sin(2 * kap * (x + t) / 3)
                          - kap * np.sin(kap * (y + t)))
    return u, ut


def _ff_error(h, n_c, T_target, u, ut, dirichlet=True):
    mats = load_fc_matrices(d=4)
    w, geo = _disk(h)
    band = WB.build_band(geo, n_c)
    nL = max(1, int(round(T_target / (n_c * h))))
    T = nL * n_c * h
    X, Y = np.meshgrid(geo.xs, geo.ys)
    gf = (lambda t: u(geo.bdry_x, geo.bdry_y, t)) if dirichlet else None
    gtf = (lambda t: ut(geo.bdry_x, geo.bdry_y, t)) if dirichlet else None
    U, Ut = V.forward_wave(geo, mats, band, 1.0, nL, u(X, Y, 0.0), ut(X, Y, 0.0), gf, gtf)
    return (np.abs(U - u(X, Y, T))[geo.inside].max(),
            np.abs(Ut - ut(X, Y, T))[geo.inside].max())


def test_plane_wave_converges():
    """Section 4.2.1, first example: u = cos(2k(x+t)/3) + cos(k(y+t)) on the unit disk
    with its Dirichlet data, n_c = 6, d = 4, k = 10.5 (15 points per wavelength at
    h = 0.04), to t = 0.48: the FF error falls at fourth order (the boundary closure's
    order) from 6.9e-3 to 3.3e-4 as h halves."""
    u, ut = _plane_wave(10.5)
    e1, _ = _ff_error(0.04, 6, 0.48, u, ut)
    e2, et2 = _ff_error(0.02, 6, 0.48, u, ut)
    assert e1 < 1e-2 and e2 < 5e-4, (e1, e2)
    assert np.log2(e1 / e2) > 3.5
    assert et2 < 5e-3 * 10.5


def test_disk_eigenmode_converges():
    """u = J_2(j r) cos(2 phi) cos(j t), j = j_{2,3} (zero Dirichlet data), n_c = 8, to
    t = 0.96: errors 1.2e-3-class at h = 0.04 falling at fourth order."""
    j = jn_zeros(2, 3)[-1]

    def u(x, y, t):
        return jv(2, j * np.hypot(x, y)) * np.cos(2 * np.arctan2(y, x)) * np.cos(j * t)

    def ut(x, y, t):
        return -j * jv(2, j * np.hypot(x, y)) * np.cos(2 * np.arctan2(y, x)) * np.sin(j * t)

    e1, _ = _ff_error(0.04, 8, 0.96, u, ut, dirichlet=False)
    e2, _ = _ff_error(0.02, 8, 0.96, u, ut, dirichlet=False)
    assert e1 < 2e-3 and e2 < 1.5e-4, (e1, e2)
    assert np.log2(e1 / e2) > 3.5


def test_zero_data_stay_zero_and_a_pulse_stays_bounded():
    """Zero initial and boundary data give zero; a Gaussian pulse (zero Dirichlet data)
    stays bounded by its initial amplitude over many large steps (no growth)."""
    mats = load_fc_matrices(d=4)
    w, geo = _disk(0.05, (0.31, 0.17))
    band = WB.build_band(geo, 6)
    X, Y = np.meshgrid(geo.xs, geo.ys)
    Z = np.zeros_like(X)
    U, Ut = V.forward_wave(geo, mats, band, 1.0, 2, Z, Z)
    assert np.abs(U).max() == 0.0 and np.abs(Ut).max() == 0.0
    f = np.exp(-((X - 0.2) ** 2 + (Y + 0.1) ** 2) / (2 * 0.1 ** 2))
    U, Ut = V.forward_wave(geo, mats, band, 1.0, 12, f, Z)  # t = 3.6
    assert np.isfinite(U).all() and np.abs(U[geo.inside]).max() < 1.0
