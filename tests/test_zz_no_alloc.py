"""fc2d_coeffs_static, the DFT entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they call: a host that
owns all device memory through its own allocator, or a loop that cannot take the
device synchronisation of cudaMalloc.  Its scratch is a fixed 64 MiB device array.
The test calls it through the C ABI (ctypes, no wrapper) twice in a row and compares
with fc2d_coeffs, within the 1e-12 bar of the DFT parity tests.  The file is named so
that pytest collects it last."""
import ctypes as ct

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_dft_matches_fc2d_coeffs_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2010_03901_gb300 import fc2d
    lib = fc2d._lib
    w = W.workload("kite160x144")
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1))
    dev = torch.device("cuda:0")
    n_f = 3
    x = torch.tensor(W.normal(21, n_f * g.ny * g.nx).reshape(n_f, g.ny, g.nx), device=dev)
    ref = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=torch.float64, device=dev)
    plan.fc2d_coeffs(n_f, x, ref)
    stream = torch.cuda.current_stream().cuda_stream
    lib.fc2d_coeffs_static.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                       ct.c_void_p]
    lib.fc2d_coeffs_static.restype = ct.c_int
    for call in range(2):
        out = torch.full_like(ref, float("nan"))
        st = lib.fc2d_coeffs_static(plan.handle, n_f, x.data_ptr(), out.data_ptr(), stream)
        assert st == 0, lib.fc2d_last_error().decode()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < 1e-12, (call, err)
    # a request above the fixed scratch is refused with an argument error
    big = lib.fc2d_coeffs_static(plan.handle, 100000, x.data_ptr(), out.data_ptr(), stream)
    assert big == 1 and b"fixed scratch" in lib.fc2d_last_error()
