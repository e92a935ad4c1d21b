"""Pins for the oracle's small-square interface procedure (Section 4.2): the placement
serves every interface point once, from a square inside the domain whose disk of
dependence holds it; a square's expansion reproduces its data; and the Fourier
Forwarding solve with square-served interface values matches the solve with the full
inverse DFT to the 1D-FC accuracy, converging as h falls, with the same error against the
exact plane wave of Section 4.2.1's first example."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle import wave as OV
from oracle import wave_boundary as OWB
from oracle import wave_squares as OWS
from oracle.fc_matrices import load_fc_matrices
from tests.fc2d_check import paper_setup


def _disk(h):
    w = paper_setup(W.disk(), h, d=4)
    g = W.Grid(a0=w.grid.a0 - 0.31 * h, b0=w.grid.b0 - 0.17 * h, h=h, nx=w.grid.nx,
               ny=w.grid.ny)
    w = W.Workload(w.name, w.boundary, g, w.params)
    return w, OG.build_geometry(w)


@pytest.mark.parametrize("h,n_c", [(0.01, 6), (0.02, 4)])
def test_placement_serves_every_interface_point_once(h, n_c):
    w, geo = _disk(h)
    band = OWB.build_band(geo, n_c, OWS.band_reach_cells(n_c))
    sq = OWS.place(geo, band.iface_lin, n_c)
    nx = geo.grid.nx
    assert sq.a == 18 and sq.R == 18 - n_c
    assert np.all(sq.owner >= 0)
    allserved = np.concatenate(sq.served)
    assert np.array_equal(np.sort(allserved), np.arange(len(band.iface_lin)))
    qj, qi = np.divmod(np.asarray(band.iface_lin), nx)
    for k, (cj, ci) in enumerate(sq.centres):
        block = geo.inside[cj - sq.a:cj + sq.a + 1, ci - sq.a:ci + sq.a + 1]
        assert block.shape == (37, 37) and block.all()
        s = sq.served[k]
        assert np.all(np.abs(qj[s] - cj) <= sq.R) and np.all(np.abs(qi[s] - ci) <= sq.R)
    # the band of this mode: interface points at least sqrt(2) n_c h from the curve
    d = band.dist.ravel()[band.iface_lin]
    assert d.min() >= np.sqrt(2) * n_c * h


def test_square_expansion_reproduces_its_data():
    """The 1D-FC continuation keeps the data at the square's points, so the expansion's
    inverse DFT at tau = 0 returns the data (to round-off), and the continuation of a
    smooth function is smooth (its spectrum decays by 1e-8 at the box's Nyquist)."""
    mats = load_fc_matrices(d=4)
    h = 0.01
    x = h * np.arange(37)
    X, Y = np.meshgrid(x, x)
    f = np.cos(3 * X + 1) * np.exp(Y)
    P = OWS.continue_2d(mats, f)
    assert P.shape == (64, 64)
    assert np.abs(P[:37, :37] - f).max() == 0.0
    c = np.abs(np.fft.fft2(P)) / 64 ** 2
    assert c[28:36, :].max() < 1e-6 * c.max() and c[:, 28:36].max() < 1e-6 * c.max()


def test_squares_match_the_full_inverse_dft_and_converge():
    """E7 (k = 10.5, n_c = 6, to t = 0.48) with square-served interface values against
    the same solve with the full inverse DFT at every small step: the two differ by
    8e-6, 6e-7 at h = 0.02, 0.01 (the squares' 1D-FC error, falling at third order or
    better) and have the same error against the exact solution (within 1%)."""
    kap, n_c = 10.5, 6
    u = lambda x, y, t: np.cos(2 * kap * (x + t) / 3) + np.cos(kap * (y + t))
    ut = lambda x, y, t: (-(2 * kap / 3) * np.sin(2 * kap * (x + t) / 3)
                          - kap * np.sin(kap * (y + t)))
    mats = load_fc_matrices(d=4)
    diffs = []
    for h in (0.02, 0.01):
        w, geo = _disk(h)
        band = OWB.build_band(geo, n_c, OWS.band_reach_cells(n_c))
        sq = OWS.place(geo, band.iface_lin, n_c)
        nL = int(round(0.48 / (n_c * h)))
        T = nL * n_c * h
        X, Y = np.meshgrid(geo.xs, geo.ys)
        gf = lambda t: u(geo.bdry_x, geo.bdry_y, t)
        gtf = lambda t: ut(geo.bdry_x, geo.bdry_y, t)
        st = OF.matching_stencils(geo)
        Ue, _ = OV.forward_wave(geo, mats, band, 1.0, nL, u(X, Y, 0), ut(X, Y, 0), gf, gtf,
                                stencils=st)
        Us, _ = OV.forward_wave(geo, mats, band, 1.0, nL, u(X, Y, 0), ut(X, Y, 0), gf, gtf,
                                stencils=st, squares=sq)
        ins = geo.inside
        ee, es = np.abs(Ue - u(X, Y, T))[ins].max(), np.abs(Us - u(X, Y, T))[ins].max()
        assert es < 1.01 * ee
        diffs.append(np.abs(Us - Ue)[ins].max())
    assert diffs[0] < 2e-5 and diffs[1] < 1.5e-6, diffs
    assert np.log2(diffs[0] / diffs[1]) > 3
