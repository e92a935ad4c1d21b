"""Plan groups (fc2d_group_extend_coeffs): several domains in one CUDA graph, the
mixed-form members' strip values from one persistent work-queue kernel, then a branch
per plan.  The spectra must equal separate fc2d_extend_coeffs calls bit for bit, on the
first call (capture), on replays over updated inputs, after a re-capture with other
buffers, with interior data only, after a member's workspace grew, and in a group of
FP64 and mixed-form plans together; the persistent kernel's tuned CTA shape is
reported."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG

pytestmark = pytest.mark.gpu

NAMES = ["disk64", "star200", "kite160x144"]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def _setup(torch, fc2d, prec, seed):
    dev = torch.device("cuda:0")
    dt = torch.float64 if prec == fc2d.FC2D_FP64 else torch.float32
    plans, fg, fb, out, ref, n_f = [], [], [], [], [], []
    for i, name in enumerate(NAMES):
        w = W.workload(name)
        g, p = w.grid, w.params
        plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                              dict(B=p.B, k1=p.k1), precision=prec)
        geo = OG.build_geometry(w)
        nf = 1 + i  # uneven function counts
        fs = [W.trig_sum(8, seed + 10 * i + k) for k in range(nf)]
        fg.append(torch.tensor(np.stack([W.grid_values(w, f) for f in fs]), device=dev))
        fb.append(torch.tensor(np.stack([OF.boundary_values(geo, f) for f in fs]), device=dev))
        out.append(torch.zeros((nf, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=dev))
        ref.append(torch.zeros_like(out[-1]))
        plans.append(plan)
        n_f.append(nf)
    return plans, fg, fb, out, ref, n_f


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_equals_separate_calls(torch_cuda, precision):
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plans, fg, fb, out, ref, n_f = _setup(torch, fc2d, prec, 3)
    grp = fc2d.fc2d_group_create(plans)
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    for i, pl in enumerate(plans):
        pl.fc2d_extend_coeffs(n_f[i], fg[i], fb[i], ref[i])
        pl.fc2d_sync_status()
    for i in range(len(plans)):
        assert torch.equal(out[i], ref[i]), i
    # replay over updated inputs (same buffers)
    for i in range(len(plans)):
        fg[i].mul_(-0.5).add_(0.25)
        fb[i].mul_(-0.5).add_(0.25)
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    for i, pl in enumerate(plans):
        pl.fc2d_extend_coeffs(n_f[i], fg[i], fb[i], ref[i])
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(out[i], ref[i]), i
    # other output buffers: captured anew
    out2 = [torch.full_like(o, 3.0) for o in out]
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out2)
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(out2[i], ref[i]), i
    grp.fc2d_group_destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_interior_data_only(torch_cuda, precision):
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plans, fg, fb, out, ref, n_f = _setup(torch, fc2d, prec, 7)
    grp = fc2d.fc2d_group_create(plans)
    grp.fc2d_group_extend_coeffs(n_f, fg, None, out)
    for i, pl in enumerate(plans):
        pl.fc2d_extend_coeffs(n_f[i], fg[i], None, ref[i])
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(out[i], ref[i]), i


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_after_a_member_workspace_grew(torch_cuda, precision):
    """A direct call with more functions on a member plan replaces that plan's workspace;
    the next group call must capture anew (the old graph holds the freed buffer) and
    still equal separate calls bit for bit."""
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plans, fg, fb, out, ref, n_f = _setup(torch, fc2d, prec, 11)
    grp = fc2d.fc2d_group_create(plans)
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    torch.cuda.synchronize()
    # four functions on plan 0 (the group gives it one): a larger workspace
    big_g = fg[0].repeat(4, 1, 1).contiguous()
    big_b = fb[0].repeat(4, 1).contiguous()
    big_o = torch.zeros((4,) + tuple(out[0].shape[1:]), dtype=out[0].dtype, device=out[0].device)
    plans[0].fc2d_extend_coeffs(4, big_g, big_b, big_o)
    torch.cuda.synchronize()
    for o in out:
        o.zero_()
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    for i, pl in enumerate(plans):
        pl.fc2d_extend_coeffs(n_f[i], fg[i], fb[i], ref[i])
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(out[i], ref[i]), i
    grp.fc2d_group_destroy()


def test_group_rejects_a_repeated_plan(torch_cuda):
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    plans, *_ = _setup(torch, fc2d, fc2d.FC2D_FP64, 13)
    with pytest.raises(RuntimeError):
        fc2d.fc2d_group_create([plans[0], plans[1], plans[0]])


def test_group_of_fp64_and_mixed_plans(torch_cuda):
    """FP64 members run their whole call on a branch, mixed-form members take their strip
    values from the persistent kernel: both equal their separate calls bit for bit."""
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    p64, fg64, fb64, out64, ref64, nf64 = _setup(torch, fc2d, fc2d.FC2D_FP64, 17)
    pmx, fgmx, fbmx, outmx, refmx, nfmx = _setup(torch, fc2d, fc2d.FC2D_MIXED, 19)
    plans = [p64[0], pmx[1], p64[2], pmx[0]]
    fg = [fg64[0], fgmx[1], fg64[2], fgmx[0]]
    fb = [fb64[0], fbmx[1], fb64[2], fbmx[0]]
    out = [out64[0], outmx[1], out64[2], outmx[0]]
    ref = [ref64[0], refmx[1], ref64[2], refmx[0]]
    n_f = [nf64[0], nfmx[1], nf64[2], nfmx[0]]
    grp = fc2d.fc2d_group_create(plans)
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    for i, pl in enumerate(plans):
        pl.fc2d_extend_coeffs(n_f[i], fg[i], fb[i], ref[i])
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(out[i], ref[i]), i
    form, threads, us = grp.fc2d_group_tuning()
    assert form in ("persistent", "branches") and threads in (256, 512)
    assert min(us.values()) > 0
    grp.fc2d_group_destroy()


@pytest.mark.parametrize("form,threads", [("persistent", 256), ("persistent", 512),
                                          ("branches", 256)])
def test_group_fixed_form_equals_separate_calls(torch_cuda, form, threads):
    """Each captured form and persistent-kernel CTA shape, fixed with
    fc2d_group_tuning_set, equals separate calls bit for bit (first call and replay);
    clearing the setting tunes again."""
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    plans, fg, fb, out, ref, n_f = _setup(torch, fc2d, fc2d.FC2D_MIXED, 29)
    for i, pl in enumerate(plans):
        pl.fc2d_extend_coeffs(n_f[i], fg[i], fb[i], ref[i])
    grp = fc2d.fc2d_group_create(plans)
    grp.fc2d_group_tuning_set(form, threads)
    for _ in range(2):
        grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
        torch.cuda.synchronize()
        for i in range(len(plans)):
            assert torch.equal(out[i], ref[i]), i
        out = [torch.full_like(o, 7.0) for o in out]
    assert grp.fc2d_group_tuning()[:2] == (form, threads)
    grp.fc2d_group_tuning_set(None)
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(out[i], ref[i]), i
    assert min(grp.fc2d_group_tuning()[2].values()) > 0
    with pytest.raises(RuntimeError):
        grp.fc2d_group_tuning_set("persistent", 128)
    grp.fc2d_group_destroy()


def test_group_tuning_without_mixed_members(torch_cuda):
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    plans, fg, fb, out, ref, n_f = _setup(torch, fc2d, fc2d.FC2D_FP64, 23)
    grp = fc2d.fc2d_group_create(plans)
    assert grp.fc2d_group_tuning()[:2] == ("branches", 0)
    grp.fc2d_group_extend_coeffs(n_f, fg, fb, out)
    torch.cuda.synchronize()
    assert grp.fc2d_group_tuning()[:2] == ("branches", 0)
    grp.fc2d_group_destroy()
