"""Pins for the oracle geometry (Sections 3.1, 3.3, 3.4): closed forms on the disk and
brute force on the star and the kite."""
import numpy as np
import pytest

import workloads as W
from oracle import geometry as G


@pytest.fixture(scope="module")
def disk_geo():
    return G.build_geometry(W.workload("disk128"))


def test_disk_crossings_closed_form(disk_geo):
    geo = disk_geo
    for j, y in enumerate(geo.ys):
        X = geo.row_cross[j]
        if abs(y) < 1 - 1e-9:
            r = np.sqrt(1 - y * y)
            assert np.allclose(X, [-r, r], atol=1e-14)
        elif abs(y) > 1 + 1e-9:
            assert len(X) == 0


def test_disk_inside_matches_x2_plus_y2(disk_geo):
    geo = disk_geo
    X, Y = np.meshgrid(geo.xs, geo.ys)
    r2 = X * X + Y * Y
    sure = np.abs(r2 - 1) > 1e-12
    assert np.array_equal(geo.inside[sure], (r2 <= 1)[sure])


def test_disk_feet_closed_form(disk_geo):
    geo = disk_geo
    g = geo.grid
    i = geo.strip_lin % g.nx
    j = geo.strip_lin // g.nx
    x, y = geo.xs[i], geo.ys[j]
    r = np.hypot(x, y)
    assert np.allclose(geo.strip_eta, r - 1, atol=1e-14)
    th = np.mod(np.arctan2(y, x), 2 * np.pi)
    dth = np.angle(np.exp(1j * (geo.strip_theta - th)))
    assert np.abs(dth).max() < 1e-13
    # the strip is every exterior point within C*k1
    width = geo.params.C * geo.params.k1
    X, Y = np.meshgrid(geo.xs, geo.ys)
    R = np.hypot(X, Y).ravel()
    expect = np.nonzero((R > 1 + 1e-12) & (R - 1 <= width - 1e-12))[0]
    assert set(expect.tolist()) <= set(geo.strip_lin.tolist())
    assert len(geo.strip_lin) - len(expect) <= 2


def test_disk_normals_are_radial(disk_geo):
    geo = disk_geo
    assert np.allclose(geo.nx_, np.cos(geo.theta_p), atol=1e-15)
    assert np.allclose(geo.ny_, np.sin(geo.theta_p), atol=1e-15)


@pytest.mark.parametrize("name", ["star200", "kite160x144"])
def test_feet_by_brute_force(name):
    w = W.workload(name)
    geo = G.build_geometry(w)
    cv = geo.curve
    g = geo.grid
    i = geo.strip_lin % g.nx
    j = geo.strip_lin // g.nx
    qx, qy = geo.xs[i], geo.ys[j]
    # orthogonality of Q - q(theta) to the tangent
    fx, fy = cv.point(geo.strip_theta)
    tx, ty = cv.x(geo.strip_theta, 1), cv.y(geo.strip_theta, 1)
    ortho = ((qx - fx) * tx + (qy - fy) * ty) / (np.hypot(tx, ty) * np.maximum(geo.strip_eta, 1e-300))
    assert np.abs(ortho).max() < 1e-10
    # the foot is the nearest point: compare with 200k samples of the curve
    sel = np.arange(0, len(qx), max(1, len(qx) // 400))
    td = 2 * np.pi * np.arange(200000) / 200000
    cx, cy = cv.point(td)
    dt = td[1]
    for s in sel:
        k = int(np.argmin(np.hypot(cx - qx[s], cy - qy[s])))
        lo, hi = td[k] - dt, td[k] + dt  # ternary search refines the sampled minimum
        dist = lambda t: float(np.hypot(cv.x(t) - qx[s], cv.y(t) - qy[s]))
        for _ in range(200):
            m1, m2 = lo + (hi - lo) / 3, hi - (hi - lo) / 3
            if dist(m1) < dist(m2):
                hi = m2
            else:
                lo = m1
        dmin = dist(0.5 * (lo + hi))
        assert abs(dmin - geo.strip_eta[s]) < 1e-12
    # Q lies on the outward normal through its foot
    nx, ny = cv.normal(geo.strip_theta)
    assert np.allclose(qx, fx + geo.strip_eta * nx, atol=1e-12)
    assert np.allclose(qy, fy + geo.strip_eta * ny, atol=1e-12)


def test_inside_against_polygon_even_odd():
    w = W.workload("kite160x144")
    geo = G.build_geometry(w)
    vx, vy = w.boundary.polygon(200000)
    X, Y = np.meshgrid(geo.xs, geo.ys)
    ref = W._inside_polygon(X.ravel(), Y.ravel(), vx, vy).reshape(X.shape)
    diff = geo.inside != ref
    # any disagreement must be within the polygon's chord error of the curve
    if diff.any():
        cv = geo.curve
        td = 2 * np.pi * np.arange(200000) / 200000
        cx, cy = cv.point(td)
        for jj, ii in zip(*np.nonzero(diff)):
            assert np.min(np.hypot(cx - X[jj, ii], cy - Y[jj, ii])) < 1e-8


def test_clockwise_input_is_reoriented():
    b = W.disk()
    cw = W.Boundary(cx=b.cx, sx=tuple(-v for v in b.sx), cy=b.cy, sy=tuple(-v for v in b.sy))
    cv = G.make_curve(cw)
    nx, ny = cv.normal(np.array([0.3]))
    assert nx[0] > 0.9  # outward at theta = 0.3


@pytest.mark.parametrize("y", [0.0, -1e-17, 1e-17, 5e-324])
def test_row_through_theta_zero_crosses_twice(y):
    """A row through the curve's point at theta = 0 (where the sample sequence closes):
    the star r = 1 + a cos 3 theta meets y = 0 at x = 1 + a and x = -(1 - a), and a row
    within rounding of y = 0 must find both crossings."""
    a = 0.1113
    cv = G.make_curve(W.star(a, 3))
    X = G.crossings(cv, "row", y, 16 * 608)
    assert len(X) == 2, X
    assert abs(X[0] + (1 - a)) < 1e-12 and abs(X[1] - (1 + a)) < 1e-12, X
