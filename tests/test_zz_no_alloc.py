"""fc2d_coeffs_static, the DFT entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they call: a host that
owns all device memory through its own allocator, or a loop that cannot take the
device synchronisation of cudaMalloc.  Its scratch is a fixed 64 MiB device array.
The test calls it through the C ABI (ctypes, no wrapper) twice in a row and compares
with fc2d_coeffs, within the bars of the DFT parity tests (1e-12 in FP64, 1e-6 in the
mixed form), on a ragged 160 x 144 grid (the generic mixed-radix kernels) and on a
1024 x 1024 grid (the power-of-two row and column kernels), in both precisions.  The
file is named so that pytest collects it last."""
import ctypes as ct

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("kite160x144", "fp64"), ("kite1024", "fp64"), ("kite1024", "mixed"),
         ("kite160x144", "mixed")]


@pytest.mark.parametrize("name,precision", CASES)
def test_static_scratch_dft_matches_fc2d_coeffs_twice(name, precision):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2010_03901_gb300 import fc2d
    lib = fc2d._lib
    w = W.workload(name)
    g, p = w.grid, w.params
    prec = fc2d.FC2D_FP64 if precision == "fp64" else fc2d.FC2D_MIXED
    bar = 1e-12 if precision == "fp64" else 1e-6
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1), precision=prec)
    dev = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    n_f = 3
    x = torch.tensor(W.normal(21, n_f * g.ny * g.nx).reshape(n_f, g.ny, g.nx), device=dev,
                     dtype=dt)
    ref = torch.zeros((n_f, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=dev)
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
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < bar, (call, err)
    # a request above the fixed scratch is refused with an argument error
    big = lib.fc2d_coeffs_static(plan.handle, 100000, x.data_ptr(), out.data_ptr(), stream)
    assert big == 1 and b"fixed scratch" in lib.fc2d_last_error()
