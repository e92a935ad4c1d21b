"""GPU Fourier Forwarding interior propagator (Section 4.2) against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import fc2d as OF
from oracle import geometry as OG
from oracle import wave as OV
from oracle.fc_matrices import load_fc_matrices

pytestmark = pytest.mark.gpu

# U_FC(t) is the extension propagated by an operator with |cos(wt)| <= 1 and
# |sin(wt)/w| <= t; its time derivative by one with |w sin(wt)| <= w_max.  Both inherit
# the 3e-11 bar of the extended grid (the blend's conditioning floor, see
# tests/test_gpu_parity.py) through those operator norms.
TOL_EXT = 3e-11


@pytest.mark.parametrize("name", ["disk128", "star200", "kite160x144"])
def test_wave_interior_parity(name):
    torch = pytest.importorskip("torch")
    from paper_2010_03901_gb300 import fc2d
    w = W.workload(name)
    g, p = w.grid, w.params
    geo = OG.build_geometry(w)
    st = OF.matching_stencils(geo)
    f0 = W.gaussian_sum(w.boundary, 4, 11, wmin=0.1, wmax=0.2)
    g0 = W.trig_sum(6, 12)
    c, t = 1.0, 0.21
    U, Ut = OV.interior_step(geo, load_fc_matrices(), W.grid_values(w, f0),
                             OF.boundary_values(geo, f0), W.grid_values(w, g0),
                             OF.boundary_values(geo, g0), c, t, st)
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1))
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.asarray(a)[None], dtype=torch.float64, device=dev)
    u_out = torch.zeros((1, g.ny, g.nx), dtype=torch.float64, device=dev)
    ut_out = torch.zeros_like(u_out)
    plan.fc2d_wave_interior(1, c, t, T(W.grid_values(w, f0)), T(OF.boundary_values(geo, f0)),
                            T(W.grid_values(w, g0)), T(OF.boundary_values(geo, g0)), u_out, ut_out)
    plan.fc2d_sync_status()
    ef = np.abs(OF.extension(geo, load_fc_matrices(), W.grid_values(w, f0),
                             OF.boundary_values(geo, f0), st)).max()
    eg = np.abs(OF.extension(geo, load_fc_matrices(), W.grid_values(w, g0),
                             OF.boundary_values(geo, g0), st)).max()
    w_max = OV.frequencies(g, c).max()
    eu = np.abs(u_out.cpu().numpy()[0] - U).max()
    et = np.abs(ut_out.cpu().numpy()[0] - Ut).max()
    assert eu < TOL_EXT * (ef + t * eg), (eu, ef, eg)
    assert et < TOL_EXT * (w_max * ef + eg), (et, w_max, ef, eg)
