"""Pins for the oracle Poisson solver (Section 4.1): closed forms of the double-layer
equation, reproduction of harmonic data, a manufactured solution, and the paper's
Table 3."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import fc2d as F
from oracle import geometry as G
from oracle import poisson as P
from oracle.fc_matrices import load_fc_matrices
from tests.fc2d_check import paper_setup

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_double_layer_of_a_constant_on_the_circle():
    """On the unit circle the kernel is -1/(4 pi) everywhere, so -phi/2 + K phi = -phi for
    a constant phi, and the interior potential of phi = 1 is -1 (Gauss)."""
    cv = G.make_curve(W.disk())
    A = P.bie_matrix(cv, 64)
    assert np.allclose(A @ np.ones(64), -np.ones(64), atol=1e-14)
    v = P.double_layer(cv, 64, np.ones(64), np.array([0.0, 0.3]), np.array([0.0, -0.5]))
    assert np.allclose(v, -1.0, atol=1e-14)


@pytest.mark.parametrize("boundary", [W.kite(0.35, 0.7), W.star(0.15, 3), W.kite(0.65, 1.5)])
def test_harmonic_data_are_reproduced(boundary):
    """For harmonic g the Laplace solution is g itself: the Nystrom solution reproduces
    e^x cos y inside to ~1e-13 with 400 nodes (super-algebraic convergence)."""
    cv = G.make_curve(boundary)
    Nb = 400
    bx, by = P.bie_points(cv, Nb)
    harm = lambda x, y: np.exp(x) * np.cos(y)
    phi = np.linalg.solve(P.bie_matrix(cv, Nb), harm(bx, by))
    pts = np.array([[0.0, 0.0], [0.3, 0.2], [-0.5, 0.1], [0.2, -0.3]])
    v = P.double_layer(cv, Nb, phi, pts[:, 0], pts[:, 1])
    assert np.abs(v - harm(pts[:, 0], pts[:, 1])).max() < 1e-12


def test_iterated_interpolation_reproduces_polynomials():
    w = W.workload("disk64")
    geo = G.build_geometry(w)
    X, Y = np.meshgrid(geo.xs, geo.ys)
    poly = lambda x, y: 1 + x ** 7 - 2 * x ** 3 * y ** 5 + y ** 7 * x ** 2
    pts = np.array([[0.31, -0.77], [-0.9, 0.2], [0.0, 1.0]])
    got = P.up_on_points(geo, poly(X, Y), pts[:, 0], pts[:, 1], 8)
    assert np.allclose(got, poly(pts[:, 0], pts[:, 1]), rtol=0, atol=1e-11)


def test_trigonometric_refinement_is_exact_for_trig_polynomials():
    t = 2 * np.pi * np.arange(24) / 24
    f = lambda t: 1 + np.cos(3 * t) - 0.5 * np.sin(11 * t) + 0.25 * np.cos(12 * t)
    fine = P.refine_density(f(t), 4)
    tf = 2 * np.pi * np.arange(96) / 96
    assert np.allclose(fine, f(tf), atol=1e-13)
    th = np.array([0.1, 2.0, 5.5])
    assert np.allclose(P.trig_interp(f(t), th), f(th), atol=1e-13)


def test_particular_solution_has_the_extension_as_laplacian():
    """Delta u_p = f^c on the periodic grid: checked with the 4th-order central
    difference Laplacian against f inside (truncation O(h^4))."""
    w = W.workload("disk128")
    geo = G.build_geometry(w)
    mats = load_fc_matrices()
    f = W.f_expsincos
    up, _ = P.particular(geo, mats, W.grid_values(w, f), F.boundary_values(geo, f))
    h = w.grid.h
    c = np.array([-1 / 12, 4 / 3, -5 / 2, 4 / 3, -1 / 12])
    lap = sum(c[k] * (np.roll(up, 2 - k, axis=1) + np.roll(up, 2 - k, axis=0)) for k in range(5))
    lap /= h * h
    X, Y = np.meshgrid(geo.xs, geo.ys)
    deep = geo.inside & (np.hypot(X, Y) < 0.8)
    assert np.abs(lap - f(X, Y))[deep].max() < 2e-3


def test_manufactured_solution_on_the_disk():
    u, f = W.u_manufactured, W.lap_u_manufactured
    mats = load_fc_matrices()
    w = paper_setup(W.disk(), 0.025)
    geo = G.build_geometry(w)
    bx, by = P.bie_points(geo.curve, w.grid.nx)
    res = P.solve(geo, mats, W.grid_values(w, f), F.boundary_values(geo, f), u(bx, by))
    X, Y = np.meshgrid(geo.xs, geo.ys)
    err = np.abs(res["u"] - u(X, Y))[geo.inside].max() / np.abs(u(X, Y)[geo.inside]).max()
    assert err < 1e-10


def test_kite_matches_paper_table3():
    """Table 3 (d = 4, M = M_P = 7): relative l2 within a factor 3 of the printed values."""
    rows = [[float(t) for t in ln.split()] for ln in open(os.path.join(GOLD,
            "paper_table3_poisson_kite.txt")) if ln.strip() and not ln.startswith("#")]
    mats = load_fc_matrices(d=4)
    u = lambda x, y: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) / (8 * np.pi ** 2)
    f = lambda x, y: -np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    for h, ref in rows:
        w = paper_setup(W.kite(0.35, 0.7), h, d=4)
        geo = G.build_geometry(w)
        bx, by = P.bie_points(geo.curve, w.grid.nx)
        res = P.solve(geo, mats, W.grid_values(w, f), F.boundary_values(geo, f), u(bx, by))
        X, Y = np.meshgrid(geo.xs, geo.ys)
        e = (res["u"] - u(X, Y))[geo.inside]
        l2 = np.sqrt(np.mean(e ** 2) / np.mean(u(X, Y)[geo.inside] ** 2))
        assert ref / 3 < l2 < ref * 3, (h, l2, ref)
