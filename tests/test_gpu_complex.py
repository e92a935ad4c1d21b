"""GPU parity of the 2D-FC of complex-valued f (fc2d_extend_coeffs_complex: the real and
imaginary parts through the real path, the full spectrum assembled from their half
spectra) against the oracle's complex extension and full DFT, with boundary data and
from interior data only.

Bars: the full spectrum holds the same numbers as the two half spectra (its upper half
by conjugation, one addition per entry), so the real path's bars apply: 1e-12 (FP64)
with boundary data, the interior-only spectrum bar (the extended grid's 2e-10 carried
through the normalised DFT) without, and 1e-6 for the mixed form."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

CASES = ["disk128", "star200", "kite160x144"]


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


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("boundary", [True, False], ids=["bdry", "interior"])
def test_complex_spectrum_parity(name, precision, boundary, fc2d, torch_cuda):
    torch = torch_cuda
    w = W.workload(name)
    g, p = w.grid, w.params
    geo = OG.build_geometry(w)
    mats = load_fc_matrices()
    pairs = [(W.f_expsincos, W.trig_sum(12, 4)), (W.gaussian_sum(w.boundary, 16, 3), W.f_expsincos)]
    n_f = len(pairs)
    fg = np.stack([np.stack([W.grid_values(w, a), W.grid_values(w, b)]) for a, b in pairs])
    fb = np.stack([np.stack([OF.boundary_values(geo, a), OF.boundary_values(geo, b)])
                   for a, b in pairs])
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    tg = torch.tensor(fg, device=dev)
    tb = torch.tensor(fb, device=dev) if boundary else None
    fhat = torch.zeros((n_f, g.ny, g.nx, 2), dtype=dt, device=dev)
    plan.fc2d_extend_coeffs_complex(n_f, tg, tb, fhat)
    plan.fc2d_sync_status()
    got = fhat.cpu().numpy().astype(np.float64)
    st = OF.matching_stencils(geo, interior=not boundary)
    for k in range(n_f):
        fc = fg[k, 0] + 1j * fg[k, 1]
        fbc = (fb[k, 0] + 1j * fb[k, 1]) if boundary else None
        ext = OF.extension_complex(geo, mats, fc, fbc, st)
        ref = OF.coefficients_complex(ext)
        if precision == "mixed":
            bar = 1e-6
        elif boundary:
            bar = 1e-12
        else:
            bar = max(1e-12, 2e-10 * np.abs(ext).max() * plan.n_strip / (g.nx * g.ny)
                      / np.abs(ref).max())
        gk = got[k][..., 0] + 1j * got[k][..., 1]
        assert rel(gk, ref) < bar, (k, rel(gk, ref), bar)


def test_real_function_gives_the_completed_half_spectrum(fc2d, torch_cuda):
    """Imaginary part zero: the full spectrum is the real path's half spectrum completed
    by Hermitian symmetry, bit for bit on its left half."""
    torch = torch_cuda
    w = W.workload("star200")
    g, p = w.grid, w.params
    geo = OG.build_geometry(w)
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1))
    dev = torch.device("cuda:0")
    re = torch.tensor(W.grid_values(w, W.f_expsincos), device=dev)
    fbr = torch.tensor(OF.boundary_values(geo, W.f_expsincos), device=dev)
    fg = torch.stack([re, torch.zeros_like(re)])[None].contiguous()
    fb = torch.stack([fbr, torch.zeros_like(fbr)])[None].contiguous()
    full = torch.zeros((1, g.ny, g.nx, 2), dtype=torch.float64, device=dev)
    half = torch.zeros((1, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=dev)
    plan.fc2d_extend_coeffs_complex(1, fg, fb, full)
    plan.fc2d_extend_coeffs(1, re[None].contiguous(), fbr[None].contiguous(), half)
    plan.fc2d_sync_status()
    assert torch.equal(full[0, :, : g.nx // 2 + 1], half[0])
    f = full[0].cpu().numpy()
    f = f[..., 0] + 1j * f[..., 1]
    m, l = np.meshgrid(np.arange(g.ny), np.arange(g.nx // 2 + 1, g.nx), indexing="ij")
    assert np.array_equal(f[m, l], np.conj(f[(-m) % g.ny, g.nx - l]))
