"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle on the
same seeded inputs.  Errors are relative max-norms ||gpu - oracle||_inf / ||oracle||_inf
per output array; geometry decisions are bit-exact.

Bars (FP64 path):
* spectrum hat f^c (eq. (3.1)), the path's result, and the DFT alone: 1e-12;
* strip values F and the extended grid: 3e-11.  The blending matrix W = A_r Q^T has
  ||W||_inf = 1.18e4, so one ulp of relative change in the matching values moves F by up
  to 9e-13, and two FP64 evaluations of the matching values in different summation
  orders already disagree on F by up to 7.3e-12 (tests/test_oracle_fc2d.py pins this floor
  on the oracle alone).  3e-11 is about four times that floor."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

TOL = 1e-12          # spectrum, DFT, interpolation from given strip values
TOL_STRIP = 3e-11    # strip values and extended grid (about 4x the conditioning floor)
CASES = ["disk64", "disk128", "star200", "kite160x144"]


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


@pytest.fixture(scope="module")
def mats():
    return load_fc_matrices()


def functions(w):
    return [W.f_expsincos, W.gaussian_sum(w.boundary, 16, 3), W.trig_sum(12, 4)]


class Case:
    def __init__(self, name, fc2d, torch):
        self.w = w = W.workload(name)
        g, p = w.grid, w.params
        self.geo = OG.build_geometry(w)
        self.st = OF.matching_stencils(self.geo)
        self.plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                                   dict(B=p.B, k1=p.k1))
        self.fs = functions(w)
        self.fg = np.stack([W.grid_values(w, f) for f in self.fs])
        self.fb = np.stack([OF.boundary_values(self.geo, f) for f in self.fs])
        dev = torch.device("cuda:0")
        self.tg = torch.tensor(self.fg, dtype=torch.float64, device=dev)
        self.tb = torch.tensor(self.fb, dtype=torch.float64, device=dev)
        self.torch = torch
        self.dev = dev


_cases = {}


@pytest.fixture(scope="module", params=CASES)
def case(request, fc2d, torch_cuda):
    if request.param not in _cases:
        _cases[request.param] = Case(request.param, fc2d, torch_cuda)
    return _cases[request.param]


def test_fc_matrices_equal_oracle(case, mats):
    Q, Ar = case.plan.fc2d_fc_matrices()
    assert np.abs(Q - mats["Q"]).max() <= 2e-16
    assert np.abs(Ar - mats["Ar"]).max() <= 4 * np.spacing(np.abs(mats["Ar"]).max())


def test_strip_set_and_feet_equal_oracle(case):
    lin, th, eta = case.plan.fc2d_strip_points()
    geo = case.geo
    assert np.array_equal(lin, geo.strip_lin)
    dth = np.angle(np.exp(1j * (th - geo.strip_theta)))
    assert np.abs(dth).max() < 1e-12
    assert np.abs(eta - geo.strip_eta).max() < 1e-13
    assert case.plan.n_inside == int(geo.inside.sum())


def test_boundary_points_equal_oracle(case):
    xy = case.plan.fc2d_boundary_points()
    assert xy.shape[0] == len(case.geo.bdry_x)
    assert np.abs(xy[:, 0] - case.geo.bdry_x).max() < 1e-13
    assert np.abs(xy[:, 1] - case.geo.bdry_y).max() < 1e-13


def test_blend_parity(case, mats):
    """Section 3.2 + eq. (2.6): strip values F[f][p][q]."""
    torch = case.torch
    p = case.w.params
    n_f = len(case.fs)
    F = torch.zeros((n_f, p.B, p.C * p.n_r + 1), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_blend(n_f, case.tg, case.tb, F)
    case.plan.fc2d_sync_status()
    got = F.cpu().numpy()
    for k in range(n_f):
        fD = OF.matching_values(case.geo, case.st, case.fg[k], case.fb[k])
        ref = OF.blend(mats, fD)
        assert rel(got[k], ref) < TOL_STRIP, k


def test_interp_parity(case, mats):
    """Section 3.4 with the oracle's strip values as input."""
    torch = case.torch
    fD = OF.matching_values(case.geo, case.st, case.fg[0], case.fb[0])
    F = OF.blend(mats, fD)
    tF = torch.tensor(F[None], dtype=torch.float64, device=case.dev)
    vals = torch.zeros((1, case.plan.n_strip), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_interp(1, tF, vals)
    case.plan.fc2d_sync_status()
    ref = OF.interpolate_strip(case.geo, F)
    assert rel(vals.cpu().numpy()[0], ref) < TOL


def test_extend_parity(case, mats):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    ext = torch.full((n_f, g.ny, g.nx), 7.0, dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend(n_f, case.tg, case.tb, ext)
    case.plan.fc2d_sync_status()
    got = ext.cpu().numpy()
    for k in range(n_f):
        ref = OF.extension(case.geo, mats, case.fg[k], case.fb[k], case.st)
        assert rel(got[k], ref) < TOL_STRIP, k
        assert np.array_equal(got[k][case.geo.inside], case.fg[k][case.geo.inside])


def test_coeffs_parity(case, mats):
    """Eq. (3.1) DFT of the oracle's extension."""
    torch = case.torch
    g = case.w.grid
    ref_ext = OF.extension(case.geo, mats, case.fg[1], case.fb[1], case.st)
    t = torch.tensor(ref_ext[None], dtype=torch.float64, device=case.dev)
    fhat = torch.zeros((1, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_coeffs(1, t, fhat)
    case.plan.fc2d_sync_status()
    got = fhat.cpu().numpy()[0]
    got = got[..., 0] + 1j * got[..., 1]
    assert rel(got, OF.coefficients(ref_ext)) < TOL


def test_extend_coeffs_parity(case, mats):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    fhat = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend_coeffs(n_f, case.tg, case.tb, fhat)
    case.plan.fc2d_sync_status()
    got = fhat.cpu().numpy()
    for k in range(n_f):
        ref = OF.coefficients(OF.extension(case.geo, mats, case.fg[k], case.fb[k], case.st))
        gk = got[k][..., 0] + 1j * got[k][..., 1]
        assert rel(gk, ref) < TOL, k


def test_values_outside_the_domain_are_ignored(case):
    torch = case.torch
    g = case.w.grid
    noisy = case.tg.clone()
    mask = torch.tensor(~case.geo.inside, device=case.dev)
    noisy[:, mask] = 1e30
    a = torch.zeros((len(case.fs), g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=case.dev)
    b = torch.zeros_like(a)
    case.plan.fc2d_extend_coeffs(len(case.fs), case.tg, case.tb, a)
    case.plan.fc2d_extend_coeffs(len(case.fs), noisy, case.tb, b)
    case.plan.fc2d_sync_status()
    assert torch.equal(a, b)


# --------------------------------------------------------------------------- #
# mixed precision: FP64 matching values and Gram coefficients, TF32 hi/lo tensor-core
# contraction with FP32 accumulation, FP32 DFT.  Bar: 1e-6 relative max-norm against
# the FP64 oracle (the mixed form's accuracy target: the TF32 hi/lo products keep about
# 2^-21 relative, the FP32 DFT about log2(N) 2^-24).
# --------------------------------------------------------------------------- #
TOL_MIXED = 1e-6
_mplans = {}


@pytest.fixture(scope="module")
def mixed(case, fc2d):
    if case.w.name not in _mplans:
        g, p = case.w.grid, case.w.params
        _mplans[case.w.name] = fc2d.fc2d_plan(case.w.boundary.arrays(),
                                              (g.a0, g.b0, g.h, g.nx, g.ny),
                                              dict(B=p.B, k1=p.k1), precision=fc2d.FC2D_MIXED)
    return _mplans[case.w.name]


def test_mixed_blend_within_1e6(case, mixed, mats):
    torch = case.torch
    p = case.w.params
    n_f = len(case.fs)
    F = torch.zeros((n_f, p.B, p.C * p.n_r + 1), dtype=torch.float32, device=case.dev)
    mixed.fc2d_blend(n_f, case.tg, case.tb, F)
    mixed.fc2d_sync_status()
    got = F.cpu().numpy().astype(np.float64)
    for k in range(n_f):
        ref = OF.blend(mats, OF.matching_values(case.geo, case.st, case.fg[k], case.fb[k]))
        assert rel(got[k], ref) < TOL_MIXED, (k, rel(got[k], ref))


def test_mixed_extend_within_1e6(case, mixed, mats):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    ext = torch.zeros((n_f, g.ny, g.nx), dtype=torch.float32, device=case.dev)
    mixed.fc2d_extend(n_f, case.tg, case.tb, ext)
    mixed.fc2d_sync_status()
    got = ext.cpu().numpy().astype(np.float64)
    for k in range(n_f):
        ref = OF.extension(case.geo, mats, case.fg[k], case.fb[k], case.st)
        assert rel(got[k], ref) < TOL_MIXED, (k, rel(got[k], ref))


def test_mixed_extend_coeffs_within_1e6(case, mixed, mats):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    fhat = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=torch.float32, device=case.dev)
    mixed.fc2d_extend_coeffs(n_f, case.tg, case.tb, fhat)
    mixed.fc2d_sync_status()
    got = fhat.cpu().numpy().astype(np.float64)
    for k in range(n_f):
        ref = OF.coefficients(OF.extension(case.geo, mats, case.fg[k], case.fb[k], case.st))
        gk = got[k][..., 0] + 1j * got[k][..., 1]
        assert rel(gk, ref) < TOL_MIXED, (k, rel(gk, ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_compact_input_equals_full_grid(case, fc2d, precision):
    """fc2d_inside_points lists the oracle's inside points in row-major order, and
    fc2d_extend_coeffs_compact on f at those points gives the spectrum of
    fc2d_extend_coeffs on the full grid bit for bit (three functions batched)."""
    torch = case.torch
    w = case.w
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = case.plan if precision == "fp64" else fc2d.fc2d_plan(
        w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny), dict(B=p.B, k1=p.k1), precision=prec)
    lin = plan.fc2d_inside_points()
    assert np.array_equal(lin, np.flatnonzero(case.geo.inside.ravel()))
    n_f = len(case.fs)
    dt = torch.float64 if precision == "fp64" else torch.float32
    full = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=case.dev)
    comp = torch.full_like(full, float("nan"))
    plan.fc2d_extend_coeffs(n_f, case.tg, case.tb, full)
    fin = case.tg.reshape(n_f, -1)[:, torch.tensor(lin, device=case.dev)].contiguous()
    plan.fc2d_extend_coeffs_compact(n_f, fin, case.tb, comp)
    plan.fc2d_sync_status()
    assert torch.equal(full, comp)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,ny,nx", [("kite2048", 4096, 2048), ("kite1024", 2048, 1024)])
def test_dft_large_power_of_two(fc2d, torch_cuda, precision, name, ny, nx):
    """The power-of-two DFT kernels at 4096 x 2048 and 2048 x 1024 (ny x nx; FP32
    columns of 4096 points as 64 x 64 passes, of 2048 as 64 x 32) on seeded random data,
    two functions batched (1025 and 513 columns: a ragged last column group):
    1e-12 (FP64) / 1e-6 (FP32) relative max-norm against numpy's FFT of the same data.
    The 4096-point FP32 columns are run with every column-pass candidate (direct form at
    16, 32, 64 columns per block, TMA form at 16, 32; the last tile holds one live
    column), each within the bar and all equal bit for bit."""
    torch = torch_cuda
    w = W.workload(name)
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0 - 0.5 * ny * g.h + 0.5 * g.ny * g.h,
                                                g.h, nx, ny), dict(B=p.B, k1=p.k1), precision=prec)
    x = W.normal(77, 2 * ny * nx).reshape(2, ny, nx)
    dt = torch.float64 if precision == "fp64" else torch.float32
    t = torch.tensor(x, dtype=dt, device="cuda:0")
    shapes = [None]
    if precision == "mixed" and ny == 4096:
        shapes = list(fc2d.Plan.TUNING_CANDIDATES)
    tol = TOL if precision == "fp64" else TOL_MIXED
    refs = [np.fft.rfft2(t.cpu().numpy().astype(np.float64)[k]) / (nx * ny) for k in range(2)]
    first = None
    for shape in shapes:
        if shape is not None:
            plan.fc2d_tuning_set(shape[1], shape[0])
        fhat = torch.full((2, ny, nx // 2 + 1, 2), float("nan"), dtype=dt, device="cuda:0")
        plan.fc2d_coeffs(2, t, fhat)
        plan.fc2d_sync_status()
        for k in range(2):
            got = fhat.cpu().numpy().astype(np.float64)[k]
            got = got[..., 0] + 1j * got[..., 1]
            assert rel(got, refs[k]) < tol, (shape, k, rel(got, refs[k]))
        if first is None:
            first = fhat
        else:
            assert torch.equal(first, fhat), shape


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ny,nx", [(1536, 768), (640, 384), (768, 1280), (384, 640)])
def test_dft_mixed_radix_sizes(fc2d, torch_cuda, precision, ny, nx):
    """The DFT at non-power-of-two sizes (64 N2 columns with N2 = 24, 10, 12, 6 and the
    mixed-radix rows) on seeded random data, two functions batched: 1e-12 (FP64) / 1e-6
    (FP32) relative max-norm against numpy's FFT of the same data."""
    torch = torch_cuda
    w = W.workload("kite1024")
    h = 3.3 / min(nx, ny)
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    # a kite plan on an ny x nx box around it (only the DFT is exercised)
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (-0.15 - 0.5 * nx * h, -0.5 * ny * h, h, nx, ny),
                          dict(B=w.params.B, k1=0.004), precision=prec)
    x = W.normal(78 + nx, 2 * ny * nx).reshape(2, ny, nx)
    dt = torch.float64 if precision == "fp64" else torch.float32
    t = torch.tensor(x, dtype=dt, device="cuda:0")
    fhat = torch.zeros((2, ny, nx // 2 + 1, 2), dtype=dt, device="cuda:0")
    plan.fc2d_coeffs(2, t, fhat)
    plan.fc2d_sync_status()
    got = fhat.cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    tol = TOL if precision == "fp64" else TOL_MIXED
    for k in range(2):
        ref = np.fft.rfft2(t[k].cpu().numpy().astype(np.float64)) / (nx * ny)
        assert rel(got[k], ref) < tol, (k, rel(got[k], ref))
