"""GPU parity of the 2D-FC from interior data only (Remark 3.2 II: no boundary values,
f_bdry NULL through the C ABI) against the oracle's interior-only reading, on the same
seeded inputs.

Bars.  Without boundary data the foot value is an extrapolation from the red stars
(normal weights up to ~3e2 in absolute sum), so two FP64 summation orders of the
matching values already move the strip values by up to ~4e-11 relative (pinned on the
oracle alone in tests/test_oracle_fc2d.py); the FP64 bar on strip values and the
extended grid is STRIP_BAR = 2e-10, five times that.  Inside the domain the grid values
are copied and must be bit-exact.  The spectrum's bar is the extended grid's carried
through the normalised DFT (STRIP_BAR max|ext| n_strip / (N_x N_y) / max|hat f|, at
least 1e-12).  The mixed form keeps its 1e-6 bar (the matching values and Gram
coefficients stay FP64 there)."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

STRIP_BAR = 2e-10
TOL = 1e-12
TOL_MIXED = 1e-6
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


class Case:
    def __init__(self, name, fc2d, torch):
        self.w = w = W.workload(name)
        g, p = w.grid, w.params
        self.mats = load_fc_matrices()
        self.geo = OG.build_geometry(w)
        self.st = OF.matching_stencils(self.geo, interior=True)
        args = (w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny), dict(B=p.B, k1=p.k1))
        self.plan = fc2d.fc2d_plan(*args)
        self.plan_mixed = fc2d.fc2d_plan(*args, precision=fc2d.FC2D_MIXED)
        self.fs = [W.f_expsincos, W.gaussian_sum(w.boundary, 16, 3), W.trig_sum(12, 4)]
        self.fg = np.stack([W.grid_values(w, f) for f in self.fs])
        dev = torch.device("cuda:0")
        self.tg = torch.tensor(self.fg, dtype=torch.float64, device=dev)
        self.torch, self.dev = torch, dev
        self.ext = [OF.extension(self.geo, self.mats, self.fg[k], None, self.st)
                    for k in range(len(self.fs))]


_cases = {}


@pytest.fixture(scope="module", params=CASES)
def case(request, fc2d, torch_cuda):
    if request.param not in _cases:
        _cases[request.param] = Case(request.param, fc2d, torch_cuda)
    return _cases[request.param]


def test_blend_parity(case):
    torch = case.torch
    p = case.w.params
    n_f = len(case.fs)
    F = torch.zeros((n_f, p.B, p.C * p.n_r + 1), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_blend(n_f, case.tg, None, F)
    case.plan.fc2d_sync_status()
    got = F.cpu().numpy()
    for k in range(n_f):
        ref = OF.blend(case.mats, OF.matching_values(case.geo, case.st, case.fg[k], None))
        assert rel(got[k], ref) < STRIP_BAR, (k, rel(got[k], ref))


def test_extend_parity(case):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    ext = torch.full((n_f, g.ny, g.nx), 7.0, dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend(n_f, case.tg, None, ext)
    case.plan.fc2d_sync_status()
    got = ext.cpu().numpy()
    for k in range(n_f):
        assert rel(got[k], case.ext[k]) < STRIP_BAR, (k, rel(got[k], case.ext[k]))
        assert np.array_equal(got[k][case.geo.inside], case.fg[k][case.geo.inside])


def _spectrum_bar(case, k, ref):
    g = case.w.grid
    return max(TOL, STRIP_BAR * np.abs(case.ext[k]).max() * case.plan.n_strip
               / (g.nx * g.ny) / np.abs(ref).max())


def test_extend_coeffs_parity(case):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    fhat = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend_coeffs(n_f, case.tg, None, fhat)
    case.plan.fc2d_sync_status()
    got = fhat.cpu().numpy()
    for k in range(n_f):
        ref = OF.coefficients(case.ext[k])
        gk = got[k][..., 0] + 1j * got[k][..., 1]
        assert rel(gk, ref) < _spectrum_bar(case, k, ref), (k, rel(gk, ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_compact_input_equals_full_grid(case, precision):
    """f at the domain's points only, without boundary data: the same spectrum bit
    for bit as the full-grid call."""
    torch = case.torch
    plan = case.plan if precision == "fp64" else case.plan_mixed
    g = case.w.grid
    n_f = len(case.fs)
    dt = torch.float64 if precision == "fp64" else torch.float32
    lin = torch.from_numpy(plan.fc2d_inside_points()).to(case.dev)
    fin = case.tg.reshape(n_f, -1)[:, lin].contiguous()
    full = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=case.dev)
    comp = torch.zeros_like(full)
    plan.fc2d_extend_coeffs(n_f, case.tg, None, full)
    plan.fc2d_extend_coeffs_compact(n_f, fin, None, comp)
    plan.fc2d_sync_status()
    assert torch.equal(full, comp)


def test_mixed_extend_coeffs_within_1e6(case):
    torch = case.torch
    g = case.w.grid
    n_f = len(case.fs)
    fhat = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=torch.float32, device=case.dev)
    case.plan_mixed.fc2d_extend_coeffs(n_f, case.tg, None, fhat)
    case.plan_mixed.fc2d_sync_status()
    got = fhat.cpu().numpy().astype(np.float64)
    for k in range(n_f):
        ref = OF.coefficients(case.ext[k])
        gk = got[k][..., 0] + 1j * got[k][..., 1]
        assert rel(gk, ref) < TOL_MIXED, (k, rel(gk, ref))


def test_boundary_data_form_is_unchanged(case):
    """With boundary values the same plan still gives the boundary-data extension."""
    torch = case.torch
    g = case.w.grid
    fb = OF.boundary_values(case.geo, case.fs[0])
    ref = OF.extension(case.geo, case.mats, case.fg[0], fb)
    ext = torch.zeros((1, g.ny, g.nx), dtype=torch.float64, device=case.dev)
    case.plan.fc2d_extend(1, case.tg[:1], torch.tensor(fb[None], device=case.dev), ext)
    case.plan.fc2d_sync_status()
    assert rel(ext.cpu().numpy()[0], ref) < 3e-11
