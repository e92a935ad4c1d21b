"""Parity at the benchmark's full size: the kite x = cos t + 0.65 cos 2t - 0.65,
y = 1.5 sin t on a 4096^2 grid with 8192 normals, f a sum of 16 Gaussians (seed 3), in
the launch configuration bench.py times (fc2d_extend_coeffs back to back on different
input and output buffers).  The whole half spectrum is compared with the
oracle's: 1e-6 (mixed), 1e-12 (FP64) relative max-norm, and the compact-input call
must give the same spectrum bit for bit."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    import bench
    from oracle import fc2d as OF
    w = W.workload("kite4096")
    f = bench.bench_functions(w, 1)[0]
    geo, st, mats = bench.oracle_setup(w)
    ref = bench.oracle_step(w, geo, st, mats, f)[0]
    fg = W.grid_values(w, f)
    fb = OF.boundary_values(geo, f)
    return torch, w, fg, fb, ref


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_spectrum(setup, precision):
    torch, w, fg, fb, ref = setup
    from paper_2010_03901_gb300 import fc2d
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    fgs = [torch.tensor(fg[None], device=dev) for _ in range(2)]
    tb = torch.tensor(fb[None], device=dev)
    outs = [torch.zeros((1, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=dev) for _ in range(3)]
    for k in range(2):
        plan.fc2d_extend_coeffs(1, fgs[k], tb, outs[k])
    lin = torch.from_numpy(plan.fc2d_inside_points()).to(dev)
    plan.fc2d_extend_coeffs_compact(1, fgs[0].reshape(1, -1)[:, lin].contiguous(), tb, outs[2])
    plan.fc2d_sync_status()
    bar = 1e-12 if precision == "fp64" else 1e-6
    for k in range(2):
        got = outs[k].cpu().numpy().astype(np.float64)[0]
        assert rel(got[..., 0] + 1j * got[..., 1], ref) < bar, k
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
