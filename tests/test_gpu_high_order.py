"""GPU parity of the FP64 path at the paper's higher orders, d = 10 and 12 with
M = d + 3 (Section 3.6; Table 1's d = 10 rows, the Poisson runs of Fig. 5), called
through the C ABI and compared with the oracle on the same seeded inputs.

Bars.  With the paper's C, Z, n_os and m_F, ||A_r Q^T||_inf is ~3e7 at d = 10 and
~3e8 at d = 12, and two FP64 summation orders of the matching values already move the
strip values F by ~2e-8 and ~3e-7 relative (pinned on the oracle alone in
tests/test_oracle_fc2d.py).  The strip-value and extended-grid bars are
STRIP_BAR[d], three times or more that floor.  Values inside the domain are copied
and must be bit-exact.  The interpolation from given strip values is as well
conditioned as at d = 5 (1e-12).  The spectrum is a normalised sum of the extended
grid, so its error is bounded by the extended grid's: a bar of
STRIP_BAR[d] * max|ext| * n_strip / (N_x N_y) / max|hat f|, and never below 1e-12."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

STRIP_BAR = {10: 1.5e-7, 12: 2e-6}
TOL = 1e-12
CASES = [("disk128", 10), ("star200", 12)]


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


@pytest.fixture(scope="module")
def fc2d():
    from paper_2010_03901_gb300 import fc2d as mod
    return mod


class Case:
    def __init__(self, name, d, fc2d, torch):
        self.w = w = W.workload(name, d=d, M=d + 3)
        self.d = d
        g, p = w.grid, w.params
        self.mats = load_fc_matrices(d)
        self.geo = OG.build_geometry(w)
        self.st = OF.matching_stencils(self.geo)
        self.plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                                   dict(d=d, M=d + 3, B=p.B, k1=p.k1))
        self.fs = [W.f_expsincos, W.gaussian_sum(w.boundary, 16, 3), W.trig_sum(12, 4)]
        self.fg = np.stack([W.grid_values(w, f) for f in self.fs])
        self.fb = np.stack([OF.boundary_values(self.geo, f) for f in self.fs])
        dev = torch.device("cuda:0")
        self.tg = torch.tensor(self.fg, dtype=torch.float64, device=dev)
        self.tb = torch.tensor(self.fb, dtype=torch.float64, device=dev)
        self.torch, self.dev = torch, dev
        self.ext = [OF.extension(self.geo, self.mats, self.fg[k], self.fb[k], self.st)
                    for k in range(len(self.fs))]


_cases = {}


@pytest.fixture(scope="module", params=CASES, ids=[f"{n}-d{d}" for n, d in CASES])
def case(request, fc2d, torch_cuda):
    if request.param not in _cases:
        _cases[request.param] = Case(*request.param, fc2d, torch_cuda)
    return _cases[request.param]


def test_plan_takes_the_paper_defaults(case):
    assert case.plan.params["d"] == case.d and case.plan.params["M"] == case.d + 3


def test_fc_matrices_equal_oracle(case):
    Q, Ar = case.plan.fc2d_fc_matrices()
    m = case.mats
    assert np.abs(Q - m["Q"]).max() <= 2e-16
    assert np.abs(Ar - m["Ar"]).max() <= 4 * np.spacing(np.abs(m["Ar"]).max())


def test_strip_set_equals_oracle(case):
    lin, th, eta = case.plan.fc2d_strip_points()
    assert np.array_equal(lin, case.geo.strip_lin)


def test_blend_parity(case):
    """Section 3.2 and eq. (2.6) with d + 3 point stencils: strip values F."""
    torch = case.torch
    p = case.w.params
    n_f = len(case.fs)
    F = torch.zeros((n_f, p.B, p.C * p.n_r + 1), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_blend(n_f, case.tg, case.tb, F)
    case.plan.fc2d_sync_status()
    got = F.cpu().numpy()
    for k in range(n_f):
        ref = OF.blend(case.mats, OF.matching_values(case.geo, case.st, case.fg[k],
                                                     case.fb[k]))
        assert rel(got[k], ref) < STRIP_BAR[case.d], (k, rel(got[k], ref))


def test_interp_parity(case):
    """Section 3.4 with M = d + 3 (13 or 15 point Lagrange in theta and eta)."""
    torch = case.torch
    F = OF.blend(case.mats, OF.matching_values(case.geo, case.st, case.fg[0], case.fb[0]))
    tF = torch.tensor(F[None], dtype=torch.float64, device=case.dev)
    vals = torch.zeros((1, case.plan.n_strip), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_interp(1, tF, vals)
    case.plan.fc2d_sync_status()
    assert rel(vals.cpu().numpy()[0], OF.interpolate_strip(case.geo, F)) < TOL


def test_extend_parity(case):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    ext = torch.full((n_f, g.ny, g.nx), 7.0, dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend(n_f, case.tg, case.tb, ext)
    case.plan.fc2d_sync_status()
    got = ext.cpu().numpy()
    for k in range(n_f):
        assert rel(got[k], case.ext[k]) < STRIP_BAR[case.d], (k, rel(got[k], case.ext[k]))
        assert np.array_equal(got[k][case.geo.inside], case.fg[k][case.geo.inside])


def test_extend_coeffs_parity(case):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    fhat = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend_coeffs(n_f, case.tg, case.tb, fhat)
    case.plan.fc2d_sync_status()
    got = fhat.cpu().numpy()
    for k in range(n_f):
        ref = OF.coefficients(case.ext[k])
        bar = max(TOL, STRIP_BAR[case.d] * np.abs(case.ext[k]).max() * case.plan.n_strip
                  / (g.nx * g.ny) / np.abs(ref).max())
        gk = got[k][..., 0] + 1j * got[k][..., 1]
        assert rel(gk, ref) < bar, (k, rel(gk, ref), bar)


def test_mixed_precision_refuses_high_order(case, fc2d):
    """The tensor-core contraction handles d <= 8: a mixed plan at d = 10 or 12 is
    refused with FC2D_ERR_UNSUPPORTED."""
    g, p = case.w.grid, case.w.params
    with pytest.raises(fc2d.Fc2dError, match="d <= 8"):
        fc2d.fc2d_plan(case.w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                       dict(d=case.d, M=case.d + 3, B=p.B, k1=p.k1),
                       precision=fc2d.FC2D_MIXED)


# --------------------------------------------------------------------------- #
# Poisson (Section 4.1) at d = 10, M = M_P = 13
# --------------------------------------------------------------------------- #
def poisson_gpu(w, f, u_ex, fc2d, torch):
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=p.d, M=p.M, B=p.B, k1=p.k1))
    plan.fc2d_poisson_plan(0)
    xy = plan.fc2d_poisson_nodes()
    bxy = plan.fc2d_boundary_points()
    dev = torch.device("cuda:0")
    fg = torch.tensor(W.grid_values(w, f)[None], device=dev)
    fb = torch.tensor(f(bxy[:, 0], bxy[:, 1])[None], device=dev)
    gn = torch.tensor(u_ex(xy[:, 0], xy[:, 1])[None], device=dev)
    u = torch.zeros_like(fg)
    phi = torch.zeros((1, len(xy)), dtype=torch.float64, device=dev)
    plan.fc2d_poisson(1, fg, fb, gn, u, phi)
    plan.fc2d_sync_status()
    return u.cpu().numpy()[0], plan


def test_poisson_parity_d10(fc2d, torch_cuda):
    """u = u_p + v at d = 10 on the disk against the oracle (manufactured u).

    Bar: the extended grid may differ from the oracle's by STRIP_BAR[10] max|ext| at
    each of the n_strip strip points, an rms difference of at most
    e = STRIP_BAR[10] max|ext| sqrt(n_strip / (N_x N_y)).  The periodic inverse
    Laplacian maps it to at most e (2.455 (L/2 pi)^2 + R^2/4) in u_p (Cauchy-Schwarz
    with sum over k != 0 of |k|^-4 = 6.027 (L/2 pi)^4 on the square lattice, plus the
    mean's (x^2 + y^2)/4 term, R the largest |x| on the grid).  v inherits at most as
    much through u_p on the curve (maximum principle).  The d = 5 bar, 1e-11, covers
    the rest."""
    from oracle import poisson as OP
    w = W.workload("disk128", d=10, M=13)
    u_ex, f = W.u_manufactured, W.lap_u_manufactured
    geo = OG.build_geometry(w)
    mats = load_fc_matrices(10)
    bx, by = OP.bie_points(geo.curve, w.grid.nx)
    fg = W.grid_values(w, f)
    ref = OP.solve(geo, mats, fg, OF.boundary_values(geo, f), u_ex(bx, by))
    u, plan = poisson_gpu(w, f, u_ex, fc2d, torch_cuda)
    g = w.grid
    ext = OF.extension(geo, mats, fg, OF.boundary_values(geo, f))
    e = STRIP_BAR[10] * np.abs(ext).max() * np.sqrt(plan.n_strip / (g.nx * g.ny))
    L = max(g.nx, g.ny) * g.h
    X, Y = np.meshgrid(geo.xs, geo.ys)
    R2 = (X ** 2 + Y ** 2).max()
    bar = 2 * e * (2.455 * (L / (2 * np.pi)) ** 2 + R2 / 4) / np.abs(ref["u"]).max() + 1e-11
    assert rel(u, ref["u"]) < bar, (rel(u, ref["u"]), bar)
    err = np.abs(u - u_ex(X, Y))[geo.inside].max() / np.abs(u_ex(X, Y)[geo.inside]).max()
    assert err < 1e-9, err


def _table4():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_table4_poisson_kite_d10.txt")
    return [[float(t) for t in ln.split()] for ln in open(path)
            if ln.strip() and not ln.startswith("#")]


def test_oscillatory_poisson_matches_paper_table4(fc2d, torch_cuda):
    """Example 4.3 / Table 4: f = -sin(40 pi x) sin(40 pi y) on the paper's kite with
    d = 10, M = M_P = 13, k1 = k2 = h, errors over the grid points inside at a distance
    > 0.2 from the curve.  Grid sizes are the smallest even 2^a 3^b 5^c holding the
    strip (the paper's are larger; the error is a property of h).  The two finer rows
    must be within a factor 3 of the printed relative l_inf and l_2 errors, with order
    above 10 between them; the coarsest row (9.3e-4, before the asymptotic regime at
    20 points per wavelength) within a factor 10."""
    from tests.fc2d_check import paper_setup
    a = 40 * np.pi
    u_ex = lambda x, y: np.sin(a * x) * np.sin(a * y) / (2 * a * a)
    f = lambda x, y: -np.sin(a * x) * np.sin(a * y)
    errs = []
    for h, _, _, ref_inf, ref_l2 in _table4():
        w = paper_setup(W.kite(0.35, 0.7), h, d=10, smooth=True)
        u, plan = poisson_gpu(w, f, u_ex, fc2d, torch_cuda)
        g = w.grid
        xs, ys = g.a0 + g.h * np.arange(g.nx), g.b0 + g.h * np.arange(g.ny)
        X, Y = np.meshgrid(xs, ys)
        far = W.far_inside(w.boundary, xs, ys, 0.2)
        ue = u_ex(X, Y)[far]
        e = (u - u_ex(X, Y))[far]
        e_inf = np.abs(e).max() / np.abs(ue).max()
        e_l2 = np.sqrt(np.mean(e ** 2) / np.mean(ue ** 2))
        errs.append((h, e_inf, e_l2))
        k = 10 if h > 4e-3 else 3
        assert ref_inf / k < e_inf < ref_inf * k, errs
        assert ref_l2 / k < e_l2 < ref_l2 * k, errs
    assert np.log2(errs[1][1] / errs[2][1]) > 10, errs
