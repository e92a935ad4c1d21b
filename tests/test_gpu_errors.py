"""Argument errors of the C ABI's calls return their status (FC2D_ERR_ARG = 1,
FC2D_ERR_UNSUPPORTED = 7) with a message and launch nothing; the plan stays usable and
its device status word reads FC2D_OK."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2010_03901_gb300 import fc2d
    w = W.workload("disk64")
    g, p = w.grid, w.params
    mk = lambda prec: fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                                     dict(B=p.B, k1=p.k1), precision=prec)
    geo = OG.build_geometry(w)
    dev = torch.device("cuda:0")
    fg = torch.tensor(W.grid_values(w, W.f_expsincos)[None], device=dev)
    fb = torch.tensor(OF.boundary_values(geo, W.f_expsincos)[None], device=dev)
    return torch, fc2d, w, mk(fc2d.FC2D_FP64), mk(fc2d.FC2D_MIXED), fg, fb


def _status(excinfo):
    return excinfo.value.status


def test_bad_function_counts_and_null_pointers(env):
    torch, fc2d, w, plan, _, fg, fb = env
    g = w.grid
    fhat = torch.zeros((1, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=fg.device)
    for n_f in (0, -3):
        with pytest.raises(fc2d.Fc2dError, match="n_f must be >= 1") as e:
            plan.fc2d_extend_coeffs(n_f, fg, fb, fhat)
        assert _status(e) == 1
    with pytest.raises(fc2d.Fc2dError, match="null pointer") as e:
        plan.fc2d_extend_coeffs(1, None, fb, fhat)
    assert _status(e) == 1
    with pytest.raises(fc2d.Fc2dError, match="null pointer"):
        plan.fc2d_extend(1, fg, fb, None)
    with pytest.raises(fc2d.Fc2dError, match="null pointer"):
        plan.fc2d_coeffs(1, None, fhat)
    # the plan still works and its status word is clear
    plan.fc2d_extend_coeffs(1, fg, fb, fhat)
    plan.fc2d_sync_status()
    assert torch.isfinite(fhat).all()


def test_unsupported_combinations(env):
    torch, fc2d, w, _, mixed, fg, fb = env
    g = w.grid
    out = torch.zeros((1, g.ny, g.nx), dtype=torch.float64, device=fg.device)
    with pytest.raises(fc2d.Fc2dError, match="FP64 plans only") as e:
        mixed.fc2d_wave_interior(1, 1.0, 0.1, fg, fb, fg, fb, out, out)
    assert _status(e) == 7
    with pytest.raises(fc2d.Fc2dError, match="c > 0") as e:
        env[3].fc2d_wave_interior(1, -1.0, 0.1, fg, fb, fg, fb, out, out)
    assert _status(e) == 1


def test_group_arguments(env):
    torch, fc2d, w, plan, _, fg, fb = env
    g = w.grid
    grp = fc2d.fc2d_group_create([plan])
    fhat = torch.zeros((1, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=fg.device)
    with pytest.raises(fc2d.Fc2dError, match="bad entry") as e:
        grp.fc2d_group_extend_coeffs([0], [fg], [fb], [fhat])
    assert _status(e) == 1
    grp.fc2d_group_extend_coeffs([1], [fg], [fb], [fhat])
    plan.fc2d_sync_status()
    grp.fc2d_group_destroy()


def test_a_stalled_device_wait_times_out_and_the_plan_stays_usable(env):
    """Failure detection on the GPU without a fault: the tensor-core kernels' bounded
    mbarrier wait, run on a barrier that nothing arrives on, gives up after its polls,
    latches FC2D_ERR_TIMEOUT (4) and returns.  fc2d_sync_status reports it once, and the
    plan then computes the same spectrum, bit for bit, as before the stall."""
    torch, fc2d, w, _, mixed, fg, fb = env
    g = w.grid
    shape = (1, g.ny, g.nx // 2 + 1, 2)
    before = torch.zeros(shape, dtype=torch.float32, device=fg.device)
    mixed.fc2d_extend_coeffs(1, fg, fb, before)
    mixed.fc2d_sync_status()
    t0 = time.perf_counter()
    mixed.fc2d_wait_selftest(1 << 12)
    with pytest.raises(fc2d.Fc2dError, match="device status latched") as e:
        mixed.fc2d_sync_status()
    elapsed = time.perf_counter() - t0
    assert _status(e) == 4
    assert elapsed < 30, elapsed
    mixed.fc2d_sync_status()  # reported once
    after = torch.zeros(shape, dtype=torch.float32, device=fg.device)
    mixed.fc2d_extend_coeffs(1, fg, fb, after)
    mixed.fc2d_sync_status()
    assert torch.equal(before, after)
    for polls in (0, (1 << 22) + 1):
        with pytest.raises(fc2d.Fc2dError, match="polls must be") as e:
            mixed.fc2d_wait_selftest(polls)
        assert _status(e) == 1
