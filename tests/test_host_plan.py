"""The library's host plan (plan.cpp), run on the CPU through tests/host_plan_harness.cpp,
against the oracle: FC matrices, inside test, strip points and feet, boundary points and
the matching stencils of Section 3.2."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle.fc_matrices import load_fc_matrices
from tests import host_plan

# name, or name:d for the paper's higher orders (M = d + 3, Section 3.6)
CASES = ["disk64", "disk128", "star200", "kite160x144", "star1024", "disk128:10",
         "star200:12"]


def case_workload(name):
    if ":" in name:
        base, d = name.split(":")
        return W.workload(base, d=int(d), M=int(d) + 3)
    return W.workload(name)


@pytest.fixture(scope="module", params=CASES)
def both(request):
    w = case_workload(request.param)
    r = host_plan.run(w)
    assert r["status"] == 0, r["error"]
    return w, r, OG.build_geometry(w)


def test_fc_matrices_in_double_double_equal_the_oracle(both):
    w, r, geo = both
    p = w.params
    m = load_fc_matrices(p.d, p.C, p.Z, p.n_os, p.n_r, p.m_F)
    assert np.array_equal(r["Q"].reshape(m["Q"].shape), m["Q"]) or \
        np.abs(r["Q"].reshape(m["Q"].shape) - m["Q"]).max() <= 2e-16
    Ar = r["Ar"].reshape(m["Ar"].shape)
    assert np.abs(Ar - m["Ar"]).max() <= 4 * np.spacing(np.abs(m["Ar"]).max())


def test_inside_intervals_equal_oracle(both):
    w, r, geo = both
    g = w.grid
    inside = np.zeros((g.ny, g.nx), bool)
    off, iv = r["row_iv_off"], r["row_iv"].reshape(-1, 2)
    for j in range(g.ny):
        for k in range(off[j], off[j + 1]):
            inside[j, iv[k, 0]:iv[k, 1] + 1] = True
    assert np.array_equal(inside, geo.inside)


def test_strip_points_equal_oracle(both):
    w, r, geo = both
    assert np.array_equal(r["strip_lin"], geo.strip_lin)
    dth = np.angle(np.exp(1j * (r["strip_theta"] - geo.strip_theta)))
    assert np.abs(dth).max() < 1e-12
    assert np.abs(r["strip_eta"] - geo.strip_eta).max() < 1e-13


def test_boundary_points_equal_oracle(both):
    w, r, geo = both
    xy = r["bdry_xy"].reshape(-1, 2)
    assert len(xy) == len(geo.bdry_x)
    assert np.abs(xy[:, 0] - geo.bdry_x).max() < 1e-13
    assert np.abs(xy[:, 1] - geo.bdry_y).max() < 1e-13


def test_matching_stencils_give_the_oracle_matching_values(both):
    w, r, geo = both
    p = w.params
    B, M, d = p.B, p.M, p.d
    f = W.f_expsincos
    fg = W.grid_values(w, f).ravel()
    fb = OF.boundary_values(geo, f)
    gidx = r["gidx"].reshape(B, M - 1, M)
    gw = r["gw"].reshape(B, M - 1, M)
    wn = r["wn"].reshape(B, d - 1, M)
    vals = np.where(gidx >= 0, fg[np.maximum(gidx, 0)], fb[np.maximum(-1 - gidx, 0)])
    stars = np.einsum("bse,bse->bs", gw, vals)
    nodes = np.concatenate([fb[:B, None], stars], axis=1)
    fD = np.einsum("bqe,be->bq", wn, nodes)
    st = OF.matching_stencils(geo)
    ref = OF.matching_values(geo, st, W.grid_values(w, f), fb)
    assert np.abs(fD - ref[:, :d - 1]).max() < 1e-13 * np.abs(ref).max()


def test_interior_stencils_give_the_oracle_matching_values(both):
    """Interior data only (Remark 3.2 II): the plan's grid-node stencils and d-row
    normal weights give the oracle's matching values, foot value included."""
    w, r, geo = both
    p = w.params
    B, M, d = p.B, p.M, p.d
    assert r["interior_ok"][0] == 1
    fg = W.grid_values(w, W.f_expsincos).ravel()
    gidx = r["gidx_i"].reshape(B, M - 1, M)
    assert np.all(gidx >= 0)
    stars = np.einsum("bse,bse->bs", r["gw_i"].reshape(B, M - 1, M), fg[gidx])
    wn = r["wn_i"].reshape(B, d, M)
    assert np.all(wn[:, :, 0] == 0)
    fD = np.einsum("bqe,be->bq", wn[:, :, 1:], stars)
    st = OF.matching_stencils(geo, interior=True)
    ref = OF.matching_values(geo, st, W.grid_values(w, W.f_expsincos), None)
    # two summation orders of sums whose terms reach (sum |wn|)(sum |gw|) max|f|: the
    # foot extrapolation's weights grow with M (about 4e3 in sum at M = 13)
    amp = np.abs(wn).sum(axis=2).max() * np.abs(r["gw_i"].reshape(B, M - 1, M)).sum(axis=2).max()
    assert np.abs(fD - ref).max() < 16 * np.finfo(float).eps * amp * np.abs(fg).max()


def test_plans_of_the_eight_star_workload():
    """The library's plan builds on all eight stars of the batched workload (several of
    them symmetric about y = 0 with a grid row on it), and on the smallest one its strip
    set and inside count equal the oracle's."""
    stars = W.stars8()
    for w in stars:
        r = host_plan.run(w)
        assert r["status"] == 0, (w.name, r["error"])
    w = min(stars, key=lambda s: s.grid.nx)
    r = host_plan.run(w)
    geo = OG.build_geometry(w)
    assert np.array_equal(np.sort(r["strip_lin"]), np.sort(geo.strip_lin))


def test_compact_stencil_indices_address_the_same_points(both):
    """The plan's compact tables (for f given at the inside points only, row by row):
    each interval's compact offset is the number of inside points before it, and every
    stencil tap's compact index addresses the same grid point as its linear index."""
    w, r, geo = both
    g = w.grid
    iv = r["row_iv"].reshape(-1, 2)
    lens = iv[:, 1] - iv[:, 0] + 1
    assert np.array_equal(r["row_iv_coff"], np.concatenate([[0], np.cumsum(lens)[:-1]]))
    inside_lin = np.flatnonzero(geo.inside.ravel())          # compact order = row major
    gi, gc = r["gidx"], r["gidx_c"]
    assert np.array_equal(gi < 0, gc < 0)
    assert np.array_equal(gc[gi < 0], gi[gi < 0])
    assert np.array_equal(inside_lin[gc[gi >= 0]], gi[gi >= 0])


def _min_max_partition(cnt, cap, n_cta):
    """Brute force: the smallest possible largest range sum over partitions of cnt into
    at most n_cta consecutive ranges of at most cap entries (dynamic programming)."""
    B = len(cnt)
    pre = np.concatenate([[0], np.cumsum(cnt)])
    INF = float("inf")
    best = np.full((n_cta + 1, B + 1), INF)
    best[0, 0] = 0
    for k in range(1, n_cta + 1):
        for e in range(1, B + 1):
            for s in range(max(0, e - cap), e):
                v = max(best[k - 1, s], pre[e] - pre[s])
                if v < best[k, e]:
                    best[k, e] = v
    return best[:, B].min()


@pytest.mark.parametrize("seed,B,cap,n_cta", [(1, 240, 57, 8), (2, 300, 57, 6), (3, 128, 20, 9)])
def test_owner_partition_is_balanced(seed, B, cap, n_cta):
    """The ranges of strip points given to the blend + interpolation CTAs cover the
    normals in order, hold at most cap normals each, number at most n_cta, and the
    largest point count equals the brute-force optimum (skewed counts, as the strip
    points per normal vary with the curvature)."""
    u = W.uniform(seed, B)
    cnt = np.floor(60 * u ** 3).astype(np.int64)
    st = host_plan.partition(cnt, cap, n_cta)
    assert st[0] == 0 and st[-1] == B
    d = np.diff(st)
    assert np.all(d >= 1) and np.all(d <= cap) and len(d) <= n_cta
    pre = np.concatenate([[0], np.cumsum(cnt)])
    assert (pre[st[1:]] - pre[st[:-1]]).max() == _min_max_partition(cnt, cap, n_cta)


# --------------------------------------------------------------------------- #
# Plan errors (the host plan code on the CPU): status and message
# --------------------------------------------------------------------------- #
def _with_grid(name, **kw):
    from dataclasses import replace
    w = W.workload(name)
    return replace(w, grid=replace(w.grid, **kw))


@pytest.mark.parametrize("grid,status,msg", [
    (dict(nx=127), 7, "nx must be even"),
    (dict(nx=126, ny=126, h=3.0 / 126), 7, "2^a 3^b 5^c"),
    (dict(a0=-1.05, b0=-1.05, h=2.1 / 128), 2, "reaches the grid edge"),
])
def test_plan_rejects_bad_grids(grid, status, msg):
    r = host_plan.run(_with_grid("disk128", **grid))
    assert r["status"] == status and msg in r["error"], r["error"]


@pytest.mark.parametrize("params", [dict(d=13, M=16), dict(d=1), dict(M=17), dict(C=1)])
def test_plan_rejects_parameters_out_of_range(params):
    r = host_plan.run(W.workload("disk128", **params))
    assert r["status"] == 1 and "parameter out of range" in r["error"], r["error"]


# --------------------------------------------------------------------------- #
# The Fourier Forwarding band (wave_band.cpp, on the CPU) against the oracle
# --------------------------------------------------------------------------- #
def _rows(off, col, w, iface_map=None):
    rows = []
    for r in range(len(off) - 1):
        d = {}
        for k in range(off[r], off[r + 1]):
            c = int(col[k])
            d[(c >> 30, c & ((1 << 30) - 1))] = w[k]
        rows.append(d)
    return rows


def _oracle_rows(mats, iface_lin):
    rows = []
    for r in range(mats["u"].shape[0]):
        d = {}
        for kind, code in (("u", 0), ("f", 1), ("g", 2)):
            m = mats[kind].getrow(r)
            for c, v in zip(m.indices, m.data):
                d[(code, int(iface_lin[c]) if kind == "f" else int(c))] = v
        rows.append(d)
    return rows


@pytest.mark.parametrize("name,n_c", [("disk64", 4), ("kite160x144", 6), ("star200", 8)])
def test_wave_band_equals_the_oracle(name, n_c):
    """U_B's sets bit for bit; second-difference and slaved-point weights within 1e-12 of
    each row's largest (the crossings, hence the boundary-polynomial nodes, come from
    independent root finders); the dissipation D = B^T B / 2 to 1e-15."""
    from oracle import wave_boundary as OWB
    w = W.workload(name, d=4, M=7)
    r = host_plan.run(w, n_c)
    assert r["status"] == 0 and r["wave_status"] == 0, (r["error"], r.get("wave_error"))
    geo = OG.build_geometry(w)
    band = OWB.build_band(geo, n_c)
    assert np.array_equal(r["wb_unknown_lin"], band.unknown_lin)
    assert np.array_equal(r["wb_slaved_lin"], band.slaved_lin)
    assert np.array_equal(np.sort(r["wb_iface_lin"]), np.sort(band.iface_lin))
    assert np.abs(r["wb_unknown_dist"] - band.dist.ravel()[band.unknown_lin]).max() < 1e-14
    near = np.nonzero((geo.inside & (band.dist < band.delta - OWB.TIE * w.grid.h)).ravel())[0]
    assert np.array_equal(r["wb_near_lin"], near)
    for nm, mats in (("L", band.L), ("S", band.S)):
        a = _rows(r[f"wb_{nm}_off"], r[f"wb_{nm}_col"], r[f"wb_{nm}_w"])
        b = _oracle_rows(mats, band.iface_lin)
        assert len(a) == len(b)
        for ra, rb in zip(a, b):
            assert set(ra) == set(rb)
            scale = max(abs(v) for v in rb.values())
            assert max(abs(ra[k] - rb[k]) for k in rb) <= 1e-12 * scale
    Bu, Bf = band.Bd["u"], band.Bd["f"]
    Du, Df = (Bu.T @ Bu / 2).toarray(), (Bu.T @ Bf / 2).toarray()
    col_of = {int(v): k for k, v in enumerate(band.iface_lin)}
    a = _rows(r["wb_D_off"], r["wb_D_col"], r["wb_D_w"])
    nnz = 0
    for ri, ra in enumerate(a):
        for (kind, idx), v in ra.items():
            ref = Du[ri, idx] if kind == 0 else Df[ri, col_of[idx]]
            assert abs(v - ref) <= 1e-15
            nnz += 1
    assert nnz == int((Du != 0).sum() + (Df != 0).sum())


@pytest.mark.parametrize("name,n_c", [("kite1024", 8)])
def test_wave_squares_equal_the_oracle(name, n_c):
    """The small-square procedure's band (deeper) and square placement of the host code
    equal the oracle's: the same squares in the same order, serving the same points."""
    from oracle import wave_boundary as OWB
    from oracle import wave_squares as OWS
    w = W.workload(name, d=4, M=7)
    r = host_plan.run(w, n_c, squares=True)
    assert r["status"] == 0 and r["wave_status"] == 0 and r["squares_status"] == 0, r
    geo = OG.build_geometry(w)
    band = OWB.build_band(geo, n_c, OWS.band_reach_cells(n_c))
    sq = OWS.place(geo, band.iface_lin, n_c)
    assert np.array_equal(r["wb_unknown_lin"], band.unknown_lin)
    assert np.array_equal(r["sq_origin_j"], sq.centres[:, 0] - sq.a)
    assert np.array_equal(r["sq_origin_i"], sq.centres[:, 1] - sq.a)
    iface = np.asarray(band.iface_lin)
    lin = np.concatenate([np.sort(iface[s]) for s in sq.served])
    assert np.array_equal(r["sq_served_lin"], lin)
    nx = w.grid.nx
    qj, qi = np.divmod(r["sq_served_lin"], nx)
    k = np.repeat(np.arange(len(sq.centres)), np.diff(r["sq_served_off"]))
    assert np.array_equal(r["sq_served_local"],
                          (qj - r["sq_origin_j"][k]) * 64 + (qi - r["sq_origin_i"][k]))
