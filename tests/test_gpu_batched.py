"""The batched eight-star workload on the GPU: 32 functions per domain in one call,
non-power-of-two grids, against the oracle on sampled functions, and the same calls
replayed from one CUDA graph."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

N_F = 32
SAMPLED = (0, 17, 31)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def setup(w, index, fc2d, torch, precision):
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=precision)
    xy = plan.fc2d_boundary_points()
    fs = W.star_functions(w, index, N_F)
    xs, ys = g.coords()
    dev = torch.device("cuda:0")
    fg = torch.tensor(np.stack([W.trig_grid(t, xs, ys) for t in fs]), device=dev)
    fb = torch.tensor(np.stack([t(xy[:, 0], xy[:, 1]) for t in fs]), device=dev)
    dt = torch.float64 if precision == fc2d.FC2D_FP64 else torch.float32
    fh = torch.zeros((N_F, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=dev)
    return plan, fs, fg, fb, fh


@pytest.fixture(scope="module")
def stars():
    return W.stars8()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx", [256, 384])
def test_batched_star_against_oracle(stars, nx, precision):
    torch = pytest.importorskip("torch")
    from paper_2010_03901_gb300 import fc2d
    index, w = next((i, s) for i, s in enumerate(stars) if s.grid.nx == nx)
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    plan, fs, fg, fb, fh = setup(w, index, fc2d, torch, prec)
    plan.fc2d_extend_coeffs(N_F, fg, fb, fh)
    plan.fc2d_sync_status()
    got = fh.cpu().numpy().astype(np.float64)
    geo = OG.build_geometry(w)
    st = OF.matching_stencils(geo)
    mats = load_fc_matrices()
    xs, ys = w.grid.coords()
    tol = 1e-12 if precision == "fp64" else 1e-6
    for m in SAMPLED:
        ref = OF.coefficients(OF.extension(geo, mats, W.trig_grid(fs[m], xs, ys),
                                           OF.boundary_values(geo, fs[m]), st))
        gm = got[m][..., 0] + 1j * got[m][..., 1]
        assert rel(gm, ref) < tol, (w.name, m, rel(gm, ref))


def test_graph_replay_equals_eager(stars):
    torch = pytest.importorskip("torch")
    from paper_2010_03901_gb300 import fc2d
    runs = []
    for nx in (256, 384):
        index, w = next((i, s) for i, s in enumerate(stars) if s.grid.nx == nx)
        runs.append(setup(w, index, fc2d, torch, fc2d.FC2D_MIXED))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for plan, _, fg, fb, fh in runs:       # eager (also sizes the workspaces)
            plan.fc2d_extend_coeffs(N_F, fg, fb, fh, s)
    s.synchronize()
    eager = [fh.clone() for *_, fh in runs]
    for *_, fh in runs:
        fh.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for plan, _, fg, fb, fh in runs:
            plan.fc2d_extend_coeffs(N_F, fg, fb, fh, s)
    graph.replay()
    torch.cuda.synchronize()
    for (plan, *_), e, (*_, fh) in zip(runs, eager, runs):
        plan.fc2d_sync_status()
        assert torch.equal(e, fh)


# --------------------------------------------------------------------------- #
# The whole eight-star workload at its full size, as bench.py times it
# --------------------------------------------------------------------------- #
FULL_DOMAINS = (3, 4, 0)   # 2048^2, 1536^2 = 2^9 3 and 640^2 = 2^7 5
FULL_SAMPLED = (0, 31)


@pytest.fixture(scope="module")
def full_group():
    """Inputs of all eight stars (32 functions each) on the device, and the oracle's
    spectra of the sampled functions on three of them."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2010_03901_gb300 import fc2d
    dev = torch.device("cuda:0")
    stars = W.stars8()
    inputs = []
    for i, w in enumerate(stars):
        g, p = w.grid, w.params
        probe = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                               dict(B=p.B, k1=p.k1))
        xy = probe.fc2d_boundary_points()
        probe.fc2d_destroy()
        fs = W.star_functions(w, i, N_F)
        xs, ys = g.coords()
        fg = torch.empty((N_F, g.ny, g.nx), dtype=torch.float64, device=dev)
        for m, t in enumerate(fs):
            fg[m].copy_(torch.from_numpy(W.trig_grid(t, xs, ys)))
        fb = torch.tensor(np.stack([t(xy[:, 0], xy[:, 1]) for t in fs]), device=dev)
        inputs.append((w, fs, fg, fb))
    mats = load_fc_matrices()
    refs, exts, geos = {}, {}, {}
    for i in FULL_DOMAINS:
        w, fs = inputs[i][0], inputs[i][1]
        geo = OG.build_geometry(w)
        geos[i] = geo
        st = OF.matching_stencils(geo)
        xs, ys = w.grid.coords()
        for m in FULL_SAMPLED:
            exts[i, m] = OF.extension(geo, mats, W.trig_grid(fs[m], xs, ys),
                                      OF.boundary_values(geo, fs[m]), st)
            refs[i, m] = OF.coefficients(exts[i, m])
    return torch, fc2d, inputs, refs, exts, geos


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_star_group_against_oracle(full_group, precision):
    """One fc2d_group_extend_coeffs call over all eight stars (256^2 to 2048^2, four of
    them not powers of two) with 32 functions each, captured and then replayed as
    bench.py times it; sampled functions of three domains against the oracle (1e-12
    FP64, 1e-6 mixed relative max-norm)."""
    torch, fc2d, inputs, refs, _, _ = full_group
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    plans, outs = [], []
    for w, fs, fg, fb in inputs:
        g, p = w.grid, w.params
        plans.append(fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                                    dict(B=p.B, k1=p.k1), precision=prec))
        outs.append(torch.zeros((N_F, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=fg.device))
    grp = fc2d.fc2d_group_create(plans)
    args = ([N_F] * 8, [x[2] for x in inputs], [x[3] for x in inputs], outs)
    for _ in range(2):  # capture, then replay
        grp.fc2d_group_extend_coeffs(*args)
    torch.cuda.synchronize()
    for pl in plans:
        pl.fc2d_sync_status()
    tol = 1e-12 if precision == "fp64" else 1e-6
    for (i, m), ref in refs.items():
        got = outs[i][m].cpu().numpy().astype(np.float64)
        gm = got[..., 0] + 1j * got[..., 1]
        assert rel(gm, ref) < tol, (inputs[i][0].name, m, rel(gm, ref))
    grp.fc2d_group_destroy()
    for pl in plans:
        pl.fc2d_destroy()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_star_extension_element_wise(full_group, precision):
    """The extended grids of the 2048^2 and 1536^2 stars point by point (fc2d_extend with
    32 functions, the function count of the batched call): sampled functions 0 and 31,
    every strip point within 3e-11 (FP64) / 1e-6 (mixed) of max|f^c| of the oracle's
    extension, inside points equal to f (FP32-rounded in the mixed form), zero
    elsewhere."""
    torch, fc2d, inputs, refs, exts, geos = full_group
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    bar = 3e-11 if precision == "fp64" else 1e-6
    for i in FULL_DOMAINS[:2]:
        w, fs, fg, fb = inputs[i]
        g, p = w.grid, w.params
        plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                              dict(B=p.B, k1=p.k1), precision=prec)
        ext = torch.full((N_F, g.ny, g.nx), 7.0, dtype=dt, device=fg.device)
        plan.fc2d_extend(N_F, fg, fb, ext)
        plan.fc2d_sync_status()
        geo = geos[i]
        strip = np.zeros(g.ny * g.nx, bool)
        strip[geo.strip_lin] = True
        strip = strip.reshape(g.ny, g.nx)
        for m in FULL_SAMPLED:
            got = ext[m].cpu().numpy().astype(np.float64)
            ref = exts[i, m]
            f_in = fg[m].cpu().numpy()
            if precision == "mixed":
                f_in = f_in.astype(np.float32).astype(np.float64)
            err = np.abs(got - ref)[strip].max() / np.abs(ref).max()
            assert err < bar, (w.name, m, err)
            assert np.array_equal(got[geo.inside], f_in[geo.inside])
            assert np.all(got[~(geo.inside | strip)] == 0.0)
        plan.fc2d_destroy()
