"""Parity at the benchmark's full size: the kite x = cos t + 0.65 cos 2t - 0.65,
y = 1.5 sin t on a 4096^2 grid with 8192 normals, f a sum of 16 Gaussians (seed 3), in
the launch configuration bench.py times (fc2d_extend_coeffs back to back on different
input and output buffers).  The whole half spectrum is compared with the
oracle's: 1e-6 (mixed), 1e-12 (FP64) relative max-norm, and the compact-input call
must give the same spectrum bit for bit.  The same from interior data only (no
boundary values) and for a complex f, and the Fourier Forwarding line's step at its
full size.  Every column-pass form and width gives the same spectrum, the TMA form
also inside a plan group's captured graph."""
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
    return torch, w, fg, fb, ref, geo, mats, st


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_spectrum(setup, precision):
    torch, w, fg, fb, ref, *_ = setup
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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_extension_element_wise(setup, precision):
    """The extended grid at 4096^2, point by point (the spectrum alone would let one
    strip point be off by O(1) within the mixed bar: a strip error e moves the
    normalised spectrum by e/N^2): every strip point within 3e-11 (FP64) / 1e-6 (mixed)
    of max|f^c| against the oracle's extension, the inside points equal to f (bit for bit
    in FP64, to FP32 rounding in the mixed form), zero elsewhere.  The strip values come
    from the same kernels (and the same CTA partition, n_f = 1) as the timed
    extend + DFT call."""
    torch, w, fg, fb, ref_spec, geo, mats, st = setup
    from oracle import fc2d as OF
    from paper_2010_03901_gb300 import fc2d
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    ext = torch.full((1, g.ny, g.nx), 7.0, dtype=dt, device=dev)
    plan.fc2d_extend(1, torch.tensor(fg[None], device=dev), torch.tensor(fb[None], device=dev), ext)
    plan.fc2d_sync_status()
    got = ext.cpu().numpy().astype(np.float64)[0]
    ref = OF.extension(geo, mats, fg, fb, st)
    scale = np.abs(ref).max()
    strip = np.zeros(g.ny * g.nx, bool)
    strip[geo.strip_lin] = True
    strip = strip.reshape(g.ny, g.nx)
    bar = 3e-11 if precision == "fp64" else 1e-6
    err = np.abs(got - ref)
    assert err[strip].max() < bar * scale, (err[strip].max() / scale)
    if precision == "fp64":
        assert np.array_equal(got[geo.inside], fg[geo.inside])
    else:
        assert np.array_equal(got[geo.inside], fg[geo.inside].astype(np.float32).astype(np.float64))
    assert np.all(got[~(geo.inside | strip)] == 0.0)
    # number of strip points off by more than the bar: none (reported if any)
    assert int((err[strip] >= bar * scale).sum()) == 0


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_strip_values_element_wise(setup, precision):
    """The strip values F[p][q] of all 8192 normals at 4096^2 (fc2d_blend) against the
    oracle's blend of its matching values: 3e-11 (FP64) / 1e-6 (mixed) relative
    max-norm, and each normal's row within the same bar of the whole array's max."""
    torch, w, fg, fb, ref_spec, geo, mats, st = setup
    from oracle import fc2d as OF
    from paper_2010_03901_gb300 import fc2d
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    F = torch.zeros((1, p.B, p.C * p.n_r + 1), dtype=dt, device=dev)
    plan.fc2d_blend(1, torch.tensor(fg[None], device=dev), torch.tensor(fb[None], device=dev), F)
    plan.fc2d_sync_status()
    got = F.cpu().numpy().astype(np.float64)[0]
    ref = OF.blend(mats, OF.matching_values(geo, st, fg, fb))
    bar = 3e-11 if precision == "fp64" else 1e-6
    per_normal = np.abs(got - ref).max(axis=1) / np.abs(ref).max()
    assert per_normal.max() < bar, (per_normal.max(), int(per_normal.argmax()))


def test_full_size_fourier_forwarding_step():
    """The Fourier Forwarding line's workload at its full size: the kite on a 2048^2
    grid with d = 4, M = 7, c = 1, Delta T = 8h, u = 32 Gaussians of width 0.05 (seed 5)
    and u_t = 0, in FP64, called back to back on the launching stream as bench.py times
    it.  U_FC and its time derivative on the whole grid against the oracle's interior
    step, with the bars of tests/test_gpu_wave.py (3e-11 of the extension's size,
    through the propagator's operator norms)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from oracle import fc2d as OF
    from oracle import geometry as OG
    from oracle import wave as OV
    from oracle.fc_matrices import load_fc_matrices
    from paper_2010_03901_gb300 import fc2d
    w = W.workload("kite2048", d=4, M=7)
    g, p = w.grid, w.params
    geo = OG.build_geometry(w)
    st = OF.matching_stencils(geo)
    mats = load_fc_matrices(4, p.C, p.Z, p.n_os, p.n_r, p.m_F)
    f0 = W.gaussian_sum(w.boundary, 32, 5, wmin=0.05, wmax=0.05, margin=0.3)
    fg, fb = W.grid_values(w, f0), OF.boundary_values(geo, f0)
    c, dT = 1.0, 8 * g.h
    U, Ut = OV.interior_step(geo, mats, fg, fb, np.zeros_like(fg), np.zeros_like(fb), c, dT, st)
    ef = np.abs(OF.extension(geo, mats, fg, fb, st)).max()

    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    dev = torch.device("cuda:0")
    u0 = torch.tensor(fg[None], device=dev)
    ub = torch.tensor(fb[None], device=dev)
    ut0, utb = torch.zeros_like(u0), torch.zeros_like(ub)
    u1, ut1 = torch.empty_like(u0), torch.empty_like(u0)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        plan.fc2d_wave_interior(1, c, dT, u0, ub, ut0, utb, u1, ut1, stream)
    plan.fc2d_sync_status(stream)
    w_max = OV.frequencies(g, c).max()
    eu = np.abs(u1.cpu().numpy()[0] - U).max()
    et = np.abs(ut1.cpu().numpy()[0] - Ut).max()
    assert eu < 3e-11 * ef, (eu, ef)
    assert et < 3e-11 * w_max * ef, (et, w_max, ef)


@pytest.fixture(scope="module")
def interior_ref(setup):
    """The oracle's spectrum of the same f from interior data only (Remark 3.2 II),
    with its extension's size and strip count for the FP64 bar."""
    from oracle import fc2d as OF
    torch, w, fg, fb, ref, geo, mats, _ = setup
    st = OF.matching_stencils(geo, interior=True)
    ext = OF.extension(geo, mats, fg, None, st)
    return OF.coefficients(ext), float(np.abs(ext).max()), len(geo.strip_lin)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_interior_data_only(setup, interior_ref, precision):
    """f_bdry NULL at the full size, called back to back as bench.py times the headline.
    Bars as in tests/test_gpu_interior.py: the interior-data strip values' 2e-10
    carried through the normalised DFT (at least 1e-12) in FP64, 1e-6 mixed."""
    torch, w, fg, fb, ref, *_ = setup
    ref_i, ext_max, n_strip = interior_ref
    from paper_2010_03901_gb300 import fc2d
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    tg = torch.tensor(fg[None], device=dev)
    outs = [torch.zeros((1, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=dev) for _ in range(2)]
    for out in outs:
        plan.fc2d_extend_coeffs(1, tg, None, out)
    plan.fc2d_sync_status()
    if precision == "fp64":
        bar = max(1e-12, 2e-10 * ext_max * n_strip / (g.nx * g.ny) / np.abs(ref_i).max())
    else:
        bar = 1e-6
    got = outs[1].cpu().numpy().astype(np.float64)[0]
    assert rel(got[..., 0] + 1j * got[..., 1], ref_i) < bar, (rel(got[..., 0] + 1j * got[..., 1], ref_i), bar)
    assert torch.equal(outs[0], outs[1])


@pytest.fixture(scope="module")
def complex_ref(setup):
    """A complex f on the same kite, f = (16 Gaussians) + i exp(sin x) cos y with its
    boundary values, and the oracle's full spectrum of it."""
    from oracle import fc2d as OF
    torch, w, fg, fb, ref, geo, mats, st = setup
    gi = W.grid_values(w, W.f_expsincos)
    bi = OF.boundary_values(geo, W.f_expsincos)
    ext = OF.extension_complex(geo, mats, fg + 1j * gi, fb + 1j * bi, st)
    return gi, bi, OF.coefficients_complex(ext)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_complex_f(setup, complex_ref, precision):
    """fc2d_extend_coeffs_complex at the full size: the whole [4096][4096] spectrum
    against the oracle's complex extension and full DFT (1e-12 FP64, 1e-6 mixed, the
    real path's bars: the full spectrum holds the two half spectra's numbers)."""
    torch, w, fg, fb, *_ = setup
    gi, bi, ref_c = complex_ref
    from paper_2010_03901_gb300 import fc2d
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    tg = torch.tensor(np.stack([fg, gi])[None], device=dev)
    tb = torch.tensor(np.stack([fb, bi])[None], device=dev)
    fhat = torch.zeros((1, g.ny, g.nx, 2), dtype=dt, device=dev)
    plan.fc2d_extend_coeffs_complex(1, tg, tb, fhat)
    plan.fc2d_sync_status()
    got = fhat.cpu().numpy().astype(np.float64)[0]
    bar = 1e-12 if precision == "fp64" else 1e-6
    assert rel(got[..., 0] + 1j * got[..., 1], ref_c) < bar


def test_column_pass_candidates_give_the_same_spectrum():
    """The 4096-point column passes run in the direct form (16, 32 or 64 columns per
    block) or the TMA-pipelined form (16 or 32); the plan-time tuner times each inside
    the plan's extension step and keeps the fastest.  Every choice computes the same
    values, so each gives the spectrum of the 16-column direct form bit for bit
    (re-running one plan's column passes with every choice through fc2d_coeffs on the
    same input, one function and three functions, the latter spanning tiles of several
    functions in the TMA form's tile order; the outputs start as NaN, so an element left
    unwritten fails)."""
    torch = pytest.importorskip("torch")
    from paper_2010_03901_gb300 import fc2d
    w = W.workload("kite4096")
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=fc2d.FC2D_MIXED)
    form, cc, us = plan.fc2d_tuning()
    assert all(t > 0 for t in us.values()), us  # every candidate ran in the step
    assert us[(form, cc)] == min(us.values())
    for n_f in (1, 3):
        x = torch.tensor(W.normal(5 + n_f, n_f * g.ny * g.nx).reshape(n_f, g.ny, g.nx),
                         dtype=torch.float32, device="cuda:0")
        outs = []
        for cand_form, width in fc2d.Plan.TUNING_CANDIDATES:
            plan.fc2d_tuning_set(width, cand_form)
            assert plan.fc2d_tuning()[:2] == (cand_form, width)
            o = torch.full((n_f, g.ny, g.nx // 2 + 1, 2), float("nan"), dtype=torch.float32,
                           device="cuda:0")
            plan.fc2d_coeffs(n_f, x, o)
            plan.fc2d_sync_status()
            outs.append(o)
        for o in outs[1:]:
            assert torch.equal(outs[0], o)
    with pytest.raises(fc2d.Fc2dError):
        plan.fc2d_tuning_set(64, "tma")


def test_tma_column_form_under_group_capture(setup):
    """The TMA-pipelined column form set on the kite 4096^2 plan, run inside a plan
    group's captured CUDA graph (first call, then a replay over a new input): the
    spectra equal separate fc2d_extend_coeffs calls in the direct form bit for bit, and
    the first equals the oracle's within the mixed bar."""
    torch, w, fg, fb, ref, geo, mats, st = setup
    from paper_2010_03901_gb300 import fc2d
    g, p = w.grid, w.params
    dev = torch.device("cuda:0")
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=fc2d.FC2D_MIXED)
    fgd = torch.tensor(fg[None], device=dev)
    fbd = torch.tensor(fb[None], device=dev)
    shape = (1, g.ny, g.nx // 2 + 1, 2)
    plan.fc2d_tuning_set(16, "tma")
    grp = fc2d.fc2d_group_create([plan])
    out = torch.full(shape, float("nan"), dtype=torch.float32, device=dev)
    grp.fc2d_group_extend_coeffs([1], [fgd], [fbd], [out])
    first = out.clone()
    fgd.mul_(-0.5)
    fbd.mul_(-0.5)
    grp.fc2d_group_extend_coeffs([1], [fgd], [fbd], [out])
    torch.cuda.synchronize()
    plan.fc2d_sync_status()
    plan.fc2d_tuning_set(32, "direct")
    sep = torch.zeros(shape, dtype=torch.float32, device=dev)
    plan.fc2d_extend_coeffs(1, fgd, fbd, sep)
    plan.fc2d_sync_status()
    assert torch.equal(out, sep)
    fgd.mul_(-2.0)
    fbd.mul_(-2.0)
    plan.fc2d_extend_coeffs(1, fgd, fbd, sep)
    plan.fc2d_sync_status()
    assert torch.equal(first, sep)
    got = first.cpu().numpy().astype(np.float64)[0]
    assert rel(got[..., 0] + 1j * got[..., 1], ref) < 1e-6
