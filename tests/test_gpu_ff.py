"""GPU Fourier Forwarding solve (Section 4.2, eq. (4.9)): U_FC combined with the
near-boundary solver U_B, through the C ABI, against the oracle on the same inputs.

* the band's sets (unknowns, slaved, interface, near points) equal the oracle's;
* one U_B small step in each mode (Taylor start, leapfrog with dissipation, time
  derivative) equals the oracle's element by element: 1e-12 relative (the operators'
  weights agree to ~2e-13 of a row's largest, the crossings being computed
  independently);
* the whole solve over several large steps equals the oracle's forward_wave at every
  grid point inside the domain, u and u_t, within the bar derived below;
* the plane wave of Section 4.2.1's first example is reproduced to the oracle's
  accuracy against the exact solution;
* the small-square procedure (interface mode 1) and its double-float evaluation (mode
  2, with the bar's addition derived at EPS_DF below) equal the oracle's solve with the
  same squares.

Bar of the whole solve.  Each large step starts with two 2D-FC extensions, whose grid
values the GPU and the oracle agree on to 3e-11 of max|f| (the blend's conditioning
floor, tests/test_gpu_parity.py), and U_FC carries that through norm-1 operators (u) and
operators of norm <= w_max (u_t, tests/test_gpu_wave.py).  U_B's stable small steps do
not amplify it.  Over n_L large steps the differences add, so u is held to
3e-11 n_L (max|u| + T max|u_t|) and u_t to 3e-11 n_L (w_max max|u| + max|u_t|)."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle import wave as OV
from oracle import wave_boundary as OWB
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

TOL_EXT = 3e-11
# Double-float small-square evaluation (interface mode 2): every interface value of a
# small step carries an error of at most EPS_DF times the field's size (each double-float
# operation ~2^-44 of its operands; a 64 x 64 transform and the advance chain ~20 of them
# per output, given a factor 3 of margin: 64 2^-44).  U_B's stable steps add the
# errors of the S n_large evaluations without amplifying them, so u moves by at most
# S n_large EPS_DF |u|, and u_t, a centred difference over 2 dt, by that over dt.  On
# power-of-two grids mode 2 also evaluates U_FC at T_{j+1} in double-float: EPS_DF |u|
# per large step for u and EPS_DF w_max |u| for u_t, inside those terms (S > 1, and
# S / dt exceeds w_max on every grid tested).
EPS_DF = 64 * 2.0 ** -44


def df_bars(double_float, S, n_large, dt, size):
    """(u, u_t) additions to the parity bars for the double-float mode."""
    if not double_float:
        return 0.0, 0.0
    e = S * n_large * EPS_DF * size
    return e, e / dt


CASES = [("disk64", 4), ("kite160x144", 6), ("star200", 8)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def _setup(name):
    from paper_2010_03901_gb300 import fc2d
    w = W.workload(name, d=4, M=7)
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    return w, plan, OG.build_geometry(w)


@pytest.mark.parametrize("name,n_c", CASES)
def test_band_sets_equal_the_oracle(torch_cuda, name, n_c):
    w, plan, geo = _setup(name)
    band = OWB.build_band(geo, n_c)
    unk, sl, iface, near = plan.fc2d_wave_band_points(n_c)
    assert np.array_equal(unk, band.unknown_lin)
    assert np.array_equal(sl, band.slaved_lin)
    assert np.array_equal(np.sort(iface), np.sort(band.iface_lin))
    ref_near = np.nonzero((geo.inside & (band.dist < band.delta - OWB.TIE * w.grid.h)).ravel())[0]
    assert np.array_equal(near, ref_near)


@pytest.mark.parametrize("name,n_c", CASES)
def test_one_small_step_each_mode(torch_cuda, name, n_c):
    """fc2d_wave_ub_step against oracle.wave_boundary.first_step / step on seeded data
    for three functions (function-minor layout on the GPU)."""
    torch = torch_cuda
    w, plan, geo = _setup(name)
    band = OWB.build_band(geo, n_c)
    g, h = w.grid, w.grid.h
    n_f, c = 3, 1.7
    Nu, nb = len(band.unknown_lin), len(geo.bdry_x)
    rnd = lambda seed, *shape: W.normal(seed, int(np.prod(shape))).reshape(shape)
    u, up, ut = rnd(31, n_f, Nu), rnd(32, n_f, Nu), rnd(33, n_f, Nu)
    grid, grid_p = rnd(34, n_f, g.ny, g.nx), rnd(35, n_f, g.ny, g.nx)
    gd = rnd(36, n_f, nb)
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    out = torch.zeros((Nu, n_f), dtype=torch.float64, device=dev)
    dt = OWB.CFL * h / c
    for mode in range(3):
        plan.fc2d_wave_ub_step(n_c, n_f, mode, c, T(u.T), T(up.T), T(ut.T), T(grid), T(grid_p),
                               T(gd), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().T
        for f in range(n_f):
            fi = grid[f].ravel()[band.iface_lin]
            fpi = grid_p[f].ravel()[band.iface_lin]
            if mode == 0:
                ref = OWB.first_step(band, h, u[f], ut[f], fi, gd[f], dt)
            else:
                ref = OWB.step(band, h, u[f], up[f], fi, fpi, gd[f])
                if mode == 2:
                    ref = (ref - up[f]) / (2 * dt)
            err = np.abs(got[f] - ref).max() / np.abs(ref).max()
            assert err < 1e-12, (mode, f, err)


def _initial(w, geo, seed):
    """u0: a Gaussian sum well inside (near zero on the curve); ut0: a trig sum."""
    f0 = W.gaussian_sum(w.boundary, 3, seed, wmin=0.1, wmax=0.2)
    g0 = W.trig_sum(4, seed + 1)
    return W.grid_values(w, f0), W.grid_values(w, g0), f0, g0


@pytest.mark.parametrize("name,n_c", CASES)
def test_forward_wave_parity(torch_cuda, name, n_c):
    """Three large steps, two functions, zero Dirichlet data; then one large step with
    time-dependent Dirichlet data (a travelling plane wave's trace on the curve)."""
    torch = torch_cuda
    w, plan, geo = _setup(name)
    band = OWB.build_band(geo, n_c)
    mats = load_fc_matrices(d=4)
    g = w.grid
    c, n_large = 1.0, 3
    dev = torch.device("cuda:0")
    U0, Ut0 = [], []
    for k in range(2):
        a, b, _, _ = _initial(w, geo, 40 + 3 * k)
        U0.append(a)
        Ut0.append(b)
    u = torch.tensor(np.stack(U0), dtype=torch.float64, device=dev)
    ut = torch.tensor(np.stack(Ut0), dtype=torch.float64, device=dev)
    plan.fc2d_forward_wave(2, c, n_c, n_large, u, ut)
    plan.fc2d_sync_status()
    got_u, got_ut = u.cpu().numpy(), ut.cpu().numpy()
    T = n_large * n_c * g.h / c
    w_max = OV.frequencies(g, c).max()
    for k in range(2):
        ref_u, ref_ut = OV.forward_wave(geo, mats, band, c, n_large, U0[k], Ut0[k])
        ins = geo.inside
        mu, mut = np.abs(ref_u[ins]).max(), np.abs(ref_ut[ins]).max()
        eu = np.abs(got_u[k][ins] - ref_u[ins]).max()
        et = np.abs(got_ut[k][ins] - ref_ut[ins]).max()
        assert eu < TOL_EXT * n_large * (mu + T * mut), (k, eu, mu, mut)
        assert et < TOL_EXT * n_large * (w_max * mu + mut), (k, et, w_max, mu, mut)
        assert np.all(got_u[k][~ins] == 0) and np.all(got_ut[k][~ins] == 0)
    # time-dependent Dirichlet data
    kap = 6.0
    ue = lambda x, y, t: np.cos(kap * (0.6 * x + 0.8 * y + t))
    ute = lambda x, y, t: -kap * np.sin(kap * (0.6 * x + 0.8 * y + t))
    S = 8 * n_c
    dt = n_c * g.h / c / S
    X, Y = np.meshgrid(geo.xs, geo.ys)
    gdir = np.stack([ue(geo.bdry_x, geo.bdry_y, m * dt) for m in range(S + 1)])[:, None, :]
    gtdir = np.stack([ute(geo.bdry_x, geo.bdry_y, j * S * dt) for j in range(2)])[:, None, :]
    u = torch.tensor(ue(X, Y, 0.0)[None], dtype=torch.float64, device=dev)
    ut = torch.tensor(ute(X, Y, 0.0)[None], dtype=torch.float64, device=dev)
    plan.fc2d_forward_wave(1, c, n_c, 1, u, ut, torch.tensor(gdir, device=dev),
                           torch.tensor(gtdir, device=dev))
    plan.fc2d_sync_status()
    ref_u, ref_ut = OV.forward_wave(geo, mats, band, c, 1, ue(X, Y, 0.0), ute(X, Y, 0.0),
                                    lambda t: ue(geo.bdry_x, geo.bdry_y, t),
                                    lambda t: ute(geo.bdry_x, geo.bdry_y, t))
    ins = geo.inside
    eu = np.abs(u.cpu().numpy()[0][ins] - ref_u[ins]).max()
    et = np.abs(ut.cpu().numpy()[0][ins] - ref_ut[ins]).max()
    Td = n_c * g.h / c
    assert eu < TOL_EXT * (1 + Td * kap), eu
    assert et < TOL_EXT * (w_max + kap), et


def test_plane_wave_against_the_exact_solution(torch_cuda):
    """Section 4.2.1, first example, on the GPU: u = cos(2k(x+t)/3) + cos(k(y+t)) on the
    unit disk, k = 10.5, h = 0.02, n_c = 6, to t = 0.48 with its Dirichlet data: the
    error against the exact solution is the oracle's (3.3e-4 there), not larger."""
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    from tests.fc2d_check import paper_setup
    kap, n_c, h = 10.5, 6, 0.02
    w = paper_setup(W.disk(), h, d=4, smooth=True)
    # a grid off the disk's symmetry lines (a line through x = 1 is tangent there)
    g = W.Grid(a0=w.grid.a0 - 0.31 * h, b0=w.grid.b0 - 0.17 * h, h=h, nx=w.grid.nx, ny=w.grid.ny)
    w = W.Workload(w.name, w.boundary, g, w.params)
    p = w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=p.M, B=p.B, k1=p.k1))
    geo = OG.build_geometry(w)
    ue = lambda x, y, t: np.cos(2 * kap * (x + t) / 3) + np.cos(kap * (y + t))
    ute = lambda x, y, t: (-(2 * kap / 3) * np.sin(2 * kap * (x + t) / 3)
                           - kap * np.sin(kap * (y + t)))
    n_large = 4
    S = 8 * n_c
    dt = n_c * h / S
    X, Y = np.meshgrid(geo.xs, geo.ys)
    dev = torch.device("cuda:0")
    gdir = np.stack([ue(geo.bdry_x, geo.bdry_y, m * dt) for m in range(n_large * S + 1)])
    gtdir = np.stack([ute(geo.bdry_x, geo.bdry_y, j * S * dt) for j in range(n_large + 1)])
    u = torch.tensor(ue(X, Y, 0.0)[None], dtype=torch.float64, device=dev)
    ut = torch.tensor(ute(X, Y, 0.0)[None], dtype=torch.float64, device=dev)
    plan.fc2d_forward_wave(1, 1.0, n_c, n_large, u, ut,
                           torch.tensor(gdir[:, None, :], device=dev),
                           torch.tensor(gtdir[:, None, :], device=dev))
    plan.fc2d_sync_status()
    T = n_large * n_c * h
    err = np.abs(u.cpu().numpy()[0] - ue(X, Y, T))[geo.inside].max()
    assert err < 5e-4, err


def test_full_size_fourier_forwarding_solve(torch_cuda):
    """The bench's FF workload at its full size, in its launch configuration: the kite at
    2048^2, d = 4, n_c = 8, 32 initial conditions in one call (a Gaussian each, seeds
    50..81), zero Dirichlet data; one large step (64 small steps).  The band's sets equal
    the oracle's; functions 0 and 31 equal the oracle's forward_wave at every grid point
    inside, within the bar of the module docstring."""
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    w = W.workload("kite2048", d=4, M=7)
    g, p = w.grid, w.params
    n_c, n_f = 8, 32
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    fs = [W.gaussian_sum(w.boundary, 1, 50 + k, wmin=0.05, wmax=0.05, margin=0.35)
          for k in range(n_f)]
    U0 = np.stack([W.grid_values(w, f) for f in fs])
    dev = torch.device("cuda:0")
    u = torch.tensor(U0, device=dev)
    ut = torch.zeros_like(u)
    plan.fc2d_forward_wave(n_f, 1.0, n_c, 1, u, ut)
    plan.fc2d_sync_status()
    got_u, got_ut = u.cpu().numpy(), ut.cpu().numpy()
    geo = OG.build_geometry(w)
    band = OWB.build_band(geo, n_c)
    unk, sl, iface, near = plan.fc2d_wave_band_points(n_c)
    assert np.array_equal(unk, band.unknown_lin) and np.array_equal(sl, band.slaved_lin)
    mats = load_fc_matrices(d=4)
    st = OF.matching_stencils(geo)
    T = n_c * g.h
    w_max = OV.frequencies(g, 1.0).max()
    ins = geo.inside
    for k in (0, n_f - 1):
        ref_u, ref_ut = OV.forward_wave(geo, mats, band, 1.0, 1, U0[k], np.zeros_like(U0[k]),
                                        stencils=st)
        mu, mut = np.abs(ref_u[ins]).max(), np.abs(ref_ut[ins]).max()
        eu = np.abs(got_u[k][ins] - ref_u[ins]).max()
        et = np.abs(got_ut[k][ins] - ref_ut[ins]).max()
        assert eu < TOL_EXT * (mu + T * mut), (k, eu, mu)
        assert et < TOL_EXT * (w_max * mu + mut), (k, et, mu, mut)


def _disk_offset(h):
    from tests.fc2d_check import paper_setup
    w = paper_setup(W.disk(), h, d=4, smooth=True)
    g = W.Grid(a0=w.grid.a0 - 0.31 * h, b0=w.grid.b0 - 0.17 * h, h=h, nx=w.grid.nx,
               ny=w.grid.ny)
    return W.Workload(w.name, w.boundary, g, w.params)


@pytest.mark.parametrize("double_float", [False, True])
def test_forward_wave_small_squares_parity(torch_cuda, double_float):
    """The small-square procedure (interface_mode 1) against the oracle's forward_wave
    with the same squares: the deeper band's sets and the squares' count, then two large
    steps of two functions with zero Dirichlet data, and one large step of the plane
    wave with its time-dependent Dirichlet data, at every inside point within the bar of
    the module docstring."""
    torch = torch_cuda
    from oracle import wave_squares as OWS
    from paper_2010_03901_gb300 import fc2d
    h, n_c = 0.01, 6
    w = _disk_offset(h)
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=p.M, B=p.B, k1=p.k1))
    geo = OG.build_geometry(w)
    band = OWB.build_band(geo, n_c, OWS.band_reach_cells(n_c))
    sq = OWS.place(geo, band.iface_lin, n_c)
    counts = plan.fc2d_wave_band_info(n_c, squares=True)
    assert counts[4] == len(sq.centres)
    unk, sl, iface, near = plan.fc2d_wave_band_points(n_c, squares=True)
    assert np.array_equal(unk, band.unknown_lin) and np.array_equal(sl, band.slaved_lin)
    mats = load_fc_matrices(d=4)
    st = OF.matching_stencils(geo)
    dev = torch.device("cuda:0")
    U0, Ut0 = [], []
    for k in range(2):
        a, b, _, _ = _initial(w, geo, 60 + 3 * k)
        U0.append(a)
        Ut0.append(b)
    n_large, c = 2, 1.0
    u = torch.tensor(np.stack(U0), device=dev)
    ut = torch.tensor(np.stack(Ut0), device=dev)
    plan.fc2d_forward_wave(2, c, n_c, n_large, u, ut, squares=True, double_float=double_float)
    plan.fc2d_sync_status()
    got_u, got_ut = u.cpu().numpy(), ut.cpu().numpy()
    T = n_large * n_c * h
    w_max = OV.frequencies(g, c).max()
    ins = geo.inside
    S = 8 * n_c
    for k in range(2):
        ref_u, ref_ut = OV.forward_wave(geo, mats, band, c, n_large, U0[k], Ut0[k],
                                        stencils=st, squares=sq)
        mu, mut = np.abs(ref_u[ins]).max(), np.abs(ref_ut[ins]).max()
        du, dut = df_bars(double_float, S, n_large, n_c * h / S / c, mu + T * mut)
        assert np.abs(got_u[k][ins] - ref_u[ins]).max() < TOL_EXT * n_large * (mu + T * mut) + du
        assert (np.abs(got_ut[k][ins] - ref_ut[ins]).max()
                < TOL_EXT * n_large * (w_max * mu + mut) + dut)
    kap = 10.5
    ue = lambda x, y, t: np.cos(2 * kap * (x + t) / 3) + np.cos(kap * (y + t))
    ute = lambda x, y, t: (-(2 * kap / 3) * np.sin(2 * kap * (x + t) / 3)
                           - kap * np.sin(kap * (y + t)))
    S = 8 * n_c
    dt = n_c * h / S
    X, Y = np.meshgrid(geo.xs, geo.ys)
    gdir = np.stack([ue(geo.bdry_x, geo.bdry_y, m * dt) for m in range(S + 1)])[:, None, :]
    gtdir = np.stack([ute(geo.bdry_x, geo.bdry_y, j * S * dt) for j in range(2)])[:, None, :]
    u = torch.tensor(ue(X, Y, 0.0)[None], device=dev)
    ut = torch.tensor(ute(X, Y, 0.0)[None], device=dev)
    plan.fc2d_forward_wave(1, c, n_c, 1, u, ut, torch.tensor(gdir, device=dev),
                           torch.tensor(gtdir, device=dev), squares=True,
                           double_float=double_float)
    plan.fc2d_sync_status()
    ref_u, ref_ut = OV.forward_wave(geo, mats, band, c, 1, ue(X, Y, 0.0), ute(X, Y, 0.0),
                                    lambda t: ue(geo.bdry_x, geo.bdry_y, t),
                                    lambda t: ute(geo.bdry_x, geo.bdry_y, t),
                                    stencils=st, squares=sq)
    du, dut = df_bars(double_float, S, 1, dt, 2 + n_c * h * kap * 2)
    assert (np.abs(u.cpu().numpy()[0][ins] - ref_u[ins]).max()
            < TOL_EXT * (2 + n_c * h * kap * 2) + du)
    assert (np.abs(ut.cpu().numpy()[0][ins] - ref_ut[ins]).max()
            < TOL_EXT * (w_max * 2 + 2 * kap) + dut)


@pytest.mark.parametrize("double_float", [False, True])
def test_full_size_small_squares_solve(torch_cuda, double_float):
    """The bench's FF workload with the small-square procedure, at full size and in the
    bench's launch configuration (kite 2048^2, n_c = 8, 32 functions, one large step):
    the squares as the oracle places them, functions 0 and 31 against the oracle's solve
    with the same squares at every inside point."""
    torch = torch_cuda
    from oracle import wave_squares as OWS
    from paper_2010_03901_gb300 import fc2d
    w = W.workload("kite2048", d=4, M=7)
    g, p = w.grid, w.params
    n_c, n_f = 8, 32
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    fs = [W.gaussian_sum(w.boundary, 1, 50 + k, wmin=0.05, wmax=0.05, margin=0.35)
          for k in range(n_f)]
    U0 = np.stack([W.grid_values(w, f) for f in fs])
    dev = torch.device("cuda:0")
    u = torch.tensor(U0, device=dev)
    ut = torch.zeros_like(u)
    plan.fc2d_forward_wave(n_f, 1.0, n_c, 1, u, ut, squares=True, double_float=double_float)
    plan.fc2d_sync_status()
    got_u, got_ut = u.cpu().numpy(), ut.cpu().numpy()
    geo = OG.build_geometry(w)
    band = OWB.build_band(geo, n_c, OWS.band_reach_cells(n_c))
    sq = OWS.place(geo, band.iface_lin, n_c)
    assert plan.fc2d_wave_band_info(n_c, squares=True)[4] == len(sq.centres)
    mats = load_fc_matrices(d=4)
    st = OF.matching_stencils(geo)
    T = n_c * g.h
    w_max = OV.frequencies(g, 1.0).max()
    ins = geo.inside
    S = 8 * n_c
    for k in (0, n_f - 1):
        ref_u, ref_ut = OV.forward_wave(geo, mats, band, 1.0, 1, U0[k], np.zeros_like(U0[k]),
                                        stencils=st, squares=sq)
        mu, mut = np.abs(ref_u[ins]).max(), np.abs(ref_ut[ins]).max()
        du, dut = df_bars(double_float, S, 1, n_c * g.h / S, np.abs(U0[k]).max() + T * mut)
        assert np.abs(got_u[k][ins] - ref_u[ins]).max() < TOL_EXT * (mu + T * mut) + du, k
        assert np.abs(got_ut[k][ins] - ref_ut[ins]).max() < TOL_EXT * (w_max * mu + mut) + dut, k


def test_double_float_mode_against_fp64_squares(torch_cuda):
    """Interface mode 2 on a power-of-two grid (the squares' evaluation and U_FC at
    T_{j+1} in double-float) against mode 1 (FP64) on the same inputs: kite 1024^2,
    n_c = 8, four functions, two large steps; u and u_t inside the domain within the
    double-float bar (df_bars, which holds the U_FC evaluation's ~2^-44 |u| too)."""
    torch = torch_cuda
    from paper_2010_03901_gb300 import fc2d
    w = W.workload("kite1024", d=4, M=7)
    g, p = w.grid, w.params
    n_c, n_f, n_large = 8, 4, 2
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    fs = [W.gaussian_sum(w.boundary, 1, 90 + k, wmin=0.05, wmax=0.05, margin=0.35)
          for k in range(n_f)]
    U0 = torch.tensor(np.stack([W.grid_values(w, f) for f in fs]), device="cuda:0")
    out = []
    for df in (False, True):
        u, ut = U0.clone(), torch.zeros_like(U0)
        plan.fc2d_forward_wave(n_f, 1.0, n_c, n_large, u, ut, squares=True, double_float=df)
        plan.fc2d_sync_status()
        out.append((u.cpu().numpy(), ut.cpu().numpy()))
    ins = OG.build_geometry(w).inside
    S = 8 * n_c
    T = n_large * n_c * g.h
    for k in range(n_f):
        (u1, t1), (u2, t2) = (out[0][0][k], out[0][1][k]), (out[1][0][k], out[1][1][k])
        size = float(U0[k].abs().max()) + T * np.abs(t1[ins]).max()
        du, dut = df_bars(True, S, n_large, n_c * g.h / S, size)
        assert np.abs(u2[ins] - u1[ins]).max() < du, k
        assert np.abs(t2[ins] - t1[ins]).max() < dut, k
        assert np.array_equal(u2[~ins], u1[~ins])
