"""Thin ctypes binding of the 2D-FC C ABI (include/fc2d.h).

Argument marshalling only: every computation runs in the CUDA library.  Device
arrays are passed as anything with a ``data_ptr()`` (torch tensors) or as integer
addresses; streams as ``torch.cuda.Stream`` objects, raw handles or None (the current
torch stream).  The names follow the C entry points.  Importing this module loads
the library and raises if it is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfc2d.so")

FC2D_FP64 = 0
FC2D_MIXED = 1

STATUS = {0: "FC2D_OK", 1: "FC2D_ERR_ARG", 2: "FC2D_ERR_GEOMETRY", 3: "FC2D_ERR_NOT_CONVERGED",
          4: "FC2D_ERR_TIMEOUT", 5: "FC2D_ERR_NOMEM", 6: "FC2D_ERR_CUDA",
          7: "FC2D_ERR_UNSUPPORTED"}


class Fc2dError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Boundary(ct.Structure):
    _fields_ = [("n_modes", ct.c_int), ("cx", ct.POINTER(ct.c_double)),
                ("sx", ct.POINTER(ct.c_double)), ("cy", ct.POINTER(ct.c_double)),
                ("sy", ct.POINTER(ct.c_double))]


class _Grid(ct.Structure):
    _fields_ = [("a0", ct.c_double), ("b0", ct.c_double), ("h", ct.c_double),
                ("nx", ct.c_int), ("ny", ct.c_int)]


class _Params(ct.Structure):
    _fields_ = [("d", ct.c_int), ("C", ct.c_int), ("Z", ct.c_int), ("n_os", ct.c_int),
                ("n_r", ct.c_int), ("M", ct.c_int), ("B", ct.c_int), ("m_F", ct.c_int),
                ("k1", ct.c_double), ("precision", ct.c_int)]


class _Info(ct.Structure):
    _fields_ = [("grid", _Grid), ("params", _Params), ("n_strip", ct.c_int64),
                ("n_inside", ct.c_int64), ("n_bdry", ct.c_int64),
                ("workspace_bytes_per_function", ct.c_int64)]


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"2D-FC CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    sigs = {
        "fc2d_plan": [ct.POINTER(_Boundary), ct.POINTER(_Grid), ct.POINTER(_Params),
                      ct.POINTER(ct.c_void_p)],
        "fc2d_plan_info": [P, ct.POINTER(_Info)],
        "fc2d_boundary_points": [P, P],
        "fc2d_fc_matrices": [P, P, P],
        "fc2d_strip_points": [P, P, P, P],
        "fc2d_blend": [P, ct.c_int, P, P, P, P],
        "fc2d_interp": [P, ct.c_int, P, P, P],
        "fc2d_extend": [P, ct.c_int, P, P, P, P],
        "fc2d_coeffs": [P, ct.c_int, P, P, P],
        "fc2d_extend_coeffs": [P, ct.c_int, P, P, P, P],
        "fc2d_inside_points": [P, P],
        "fc2d_extend_coeffs_compact": [P, ct.c_int, P, P, P, P],
        "fc2d_extend_coeffs_complex": [P, ct.c_int, P, P, P, P],
        "fc2d_group_create": [P, ct.c_int, P],
        "fc2d_group_extend_coeffs": [P, P, P, P, P, P],
        "fc2d_coeffs_static": [P, ct.c_int, P, P, P],
        "fc2d_sync_status": [P, P],
        "fc2d_wait_selftest": [P, ct.c_uint32, P],
        "fc2d_poisson_plan": [P, ct.c_int],
        "fc2d_poisson_nodes": [P, P, P],
        "fc2d_poisson_info": [P, P, P, P],
        "fc2d_poisson": [P, ct.c_int, P, P, P, P, P, P],
        "fc2d_wave_interior": [P, ct.c_int, ct.c_double, ct.c_double, P, P, P, P, P, P, P],
        "fc2d_forward_wave": [P, ct.c_int, ct.c_double, ct.c_int, ct.c_int, ct.c_int, P, P, P,
                              P, P],
        "fc2d_wave_band_info": [P, ct.c_int, ct.c_int, P],
        "fc2d_wave_band_points": [P, ct.c_int, ct.c_int, P, P, P, P],
        "fc2d_wave_ub_step": [P, ct.c_int, ct.c_int, ct.c_int, ct.c_double, P, P, P, P, P, P,
                              P, P],
        "fc2d_profile": [P, ct.c_int],
        "fc2d_probe_fp64": [P, ct.c_int, ct.c_int64, P, P],
        "fc2d_tuning": [P, P, P],
        "fc2d_tuning_set": [P, P],
        "fc2d_group_tuning": [P, P, P],
        "fc2d_group_tuning_set": [P, P],
        "fc2d_profile_read": [P, ct.c_int, P, P, P, P],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ct.c_int
    lib.fc2d_destroy.argtypes = [P]
    lib.fc2d_destroy.restype = None
    lib.fc2d_group_destroy.argtypes = [P]
    lib.fc2d_group_destroy.restype = None
    lib.fc2d_last_error.argtypes = []
    lib.fc2d_last_error.restype = ct.c_char_p
    return lib


_lib = load_library()


def _check(status):
    if status != 0:
        raise Fc2dError(status, _lib.fc2d_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


class Plan:
    """An fc2d plan: geometry, FC matrices and stencils for one domain and grid."""

    def __init__(self, boundary, grid, params=None, precision=FC2D_FP64):
        cx, sx, cy, sy = (np.ascontiguousarray(a, dtype=np.float64) for a in boundary)
        self._keep = (cx, sx, cy, sy)
        dp = ct.POINTER(ct.c_double)
        b = _Boundary(len(cx), cx.ctypes.data_as(dp), sx.ctypes.data_as(dp),
                      cy.ctypes.data_as(dp), sy.ctypes.data_as(dp))
        a0, b0, h, nx, ny = grid
        g = _Grid(a0, b0, h, nx, ny)
        prm = dict(params or {})
        p = _Params(prm.get("d", 0), prm.get("C", 0), prm.get("Z", 0), prm.get("n_os", 0),
                    prm.get("n_r", 0), prm.get("M", 0), prm.get("B", 0), prm.get("m_F", 0),
                    prm.get("k1", 0.0), precision)
        h_ = ct.c_void_p()
        _check(_lib.fc2d_plan(ct.byref(b), ct.byref(g), ct.byref(p), ct.byref(h_)))
        self.handle = h_
        self.precision = precision
        inf = _Info()
        _check(_lib.fc2d_plan_info(self.handle, ct.byref(inf)))
        self.nx, self.ny = inf.grid.nx, inf.grid.ny
        self.n_strip, self.n_inside, self.n_bdry = inf.n_strip, inf.n_inside, inf.n_bdry
        pr = inf.params
        self.params = dict(d=pr.d, C=pr.C, Z=pr.Z, n_os=pr.n_os, n_r=pr.n_r, M=pr.M, B=pr.B,
                           m_F=pr.m_F, k1=pr.k1)
        self.workspace_bytes_per_function = inf.workspace_bytes_per_function

    # host queries -------------------------------------------------------------
    def fc2d_boundary_points(self):
        out = np.zeros((self.n_bdry, 2))
        _check(_lib.fc2d_boundary_points(self.handle, out.ctypes.data))
        return out

    def fc2d_fc_matrices(self):
        d, Cr = self.params["d"], self.params["C"] * self.params["n_r"]
        Q = np.zeros((d, d))
        Ar = np.zeros((Cr, d))
        _check(_lib.fc2d_fc_matrices(self.handle, Q.ctypes.data, Ar.ctypes.data))
        return Q, Ar

    def fc2d_strip_points(self):
        n = self.n_strip
        lin = np.zeros(n, np.int32)
        th = np.zeros(n)
        eta = np.zeros(n)
        _check(_lib.fc2d_strip_points(self.handle, lin.ctypes.data, th.ctypes.data,
                                      eta.ctypes.data))
        return lin, th, eta

    # device computations ----------------------------------------------------------
    def fc2d_blend(self, n_f, f_grid, f_bdry, F, stream=None):
        _check(_lib.fc2d_blend(self.handle, n_f, _ptr(f_grid), _ptr(f_bdry), _ptr(F),
                               _stream(stream)))

    def fc2d_interp(self, n_f, F, vals, stream=None):
        _check(_lib.fc2d_interp(self.handle, n_f, _ptr(F), _ptr(vals), _stream(stream)))

    def fc2d_extend(self, n_f, f_grid, f_bdry, ext, stream=None):
        _check(_lib.fc2d_extend(self.handle, n_f, _ptr(f_grid), _ptr(f_bdry), _ptr(ext),
                                _stream(stream)))

    def fc2d_coeffs(self, n_f, ext, fhat, stream=None):
        _check(_lib.fc2d_coeffs(self.handle, n_f, _ptr(ext), _ptr(fhat), _stream(stream)))

    def fc2d_extend_coeffs(self, n_f, f_grid, f_bdry, fhat, stream=None):
        _check(_lib.fc2d_extend_coeffs(self.handle, n_f, _ptr(f_grid), _ptr(f_bdry),
                                       _ptr(fhat), _stream(stream)))

    def fc2d_inside_points(self):
        """Linear indices j * nx + i of the domain's grid points, in compact order."""
        out = np.zeros(self.n_inside, dtype=np.int64)
        _check(_lib.fc2d_inside_points(self.handle, out.ctypes.data))
        return out

    def fc2d_extend_coeffs_compact(self, n_f, f_inside, f_bdry, fhat, stream=None):
        _check(_lib.fc2d_extend_coeffs_compact(self.handle, n_f, _ptr(f_inside), _ptr(f_bdry),
                                               _ptr(fhat), _stream(stream)))

    def fc2d_extend_coeffs_complex(self, n_f, f_grid, f_bdry, fhat, stream=None):
        """Complex f: f_grid [n_f][2][ny][nx] (re, im), f_bdry [n_f][2][n_bdry] or None;
        fhat [n_f][ny][nx][2] receives the full spectrum."""
        _check(_lib.fc2d_extend_coeffs_complex(self.handle, n_f, _ptr(f_grid), _ptr(f_bdry),
                                               _ptr(fhat), _stream(stream)))

    def fc2d_coeffs_static(self, n_f, ext, fhat, stream=None):
        """fc2d_coeffs without any device allocation (fixed 64 MiB scratch)."""
        _check(_lib.fc2d_coeffs_static(self.handle, n_f, _ptr(ext), _ptr(fhat),
                                       _stream(stream)))

    def fc2d_poisson_plan(self, n_b=0):
        _check(_lib.fc2d_poisson_plan(self.handle, n_b))

    def fc2d_poisson_nodes(self):
        n = ct.c_int()
        _check(_lib.fc2d_poisson_nodes(self.handle, None, ct.byref(n)))
        xy = np.zeros((n.value, 2))
        _check(_lib.fc2d_poisson_nodes(self.handle, xy.ctypes.data, ct.byref(n)))
        return xy

    def fc2d_poisson(self, n_f, f_grid, f_bdry, g_nodes, u, phi=None, stream=None):
        _check(_lib.fc2d_poisson(self.handle, n_f, _ptr(f_grid), _ptr(f_bdry), _ptr(g_nodes),
                                 _ptr(u), _ptr(phi), _stream(stream)))

    def fc2d_poisson_info(self):
        it, res, nn = ct.c_int(), ct.c_double(), ct.c_int64()
        _check(_lib.fc2d_poisson_info(self.handle, ct.byref(it), ct.byref(res), ct.byref(nn)))
        return {"gmres_iters": it.value, "gmres_resid": res.value, "n_near": nn.value}

    def fc2d_wave_interior(self, n_f, c, t, u0, u0_bdry, ut0, ut0_bdry, u_out, ut_out,
                           stream=None):
        _check(_lib.fc2d_wave_interior(self.handle, n_f, c, t, _ptr(u0), _ptr(u0_bdry),
                                       _ptr(ut0), _ptr(ut0_bdry), _ptr(u_out), _ptr(ut_out),
                                       _stream(stream)))

    def fc2d_forward_wave(self, n_f, c, n_c, n_large, u, ut, g_dir=None, gt_dir=None,
                          stream=None, squares=False, double_float=False):
        """squares: the interface values from the small-square procedure (mode 1);
        with double_float, its small-step evaluation in double-float arithmetic (mode 2)."""
        mode = (2 if double_float else 1) if squares else 0
        _check(_lib.fc2d_forward_wave(self.handle, n_f, c, n_c, n_large, mode,
                                      _ptr(u), _ptr(ut), _ptr(g_dir), _ptr(gt_dir),
                                      _stream(stream)))

    def fc2d_wave_band_info(self, n_c, squares=False):
        """(unknowns, slaved, interface, near, squares) counts of U_B's band for n_c."""
        counts = np.zeros(5, np.int64)
        _check(_lib.fc2d_wave_band_info(self.handle, n_c, 1 if squares else 0,
                                        counts.ctypes.data))
        return tuple(int(v) for v in counts)

    def fc2d_wave_band_points(self, n_c, squares=False):
        """Grid linear indices of the unknowns, slaved, interface and near points."""
        n = self.fc2d_wave_band_info(n_c, squares)[:4]
        arrs = [np.zeros(max(k, 1), np.int32) for k in n]
        _check(_lib.fc2d_wave_band_points(self.handle, n_c, 1 if squares else 0,
                                          *[a.ctypes.data for a in arrs]))
        return [a[:k] for a, k in zip(arrs, n)]

    def fc2d_wave_ub_step(self, n_c, n_f, mode, c, u, u_prev, ut, grid, grid_prev, g, out,
                          stream=None):
        _check(_lib.fc2d_wave_ub_step(self.handle, n_c, n_f, mode, c, _ptr(u), _ptr(u_prev),
                                      _ptr(ut), _ptr(grid), _ptr(grid_prev), _ptr(g), _ptr(out),
                                      _stream(stream)))

    # the column-pass candidates the plan-time tuner times, in the order of its times
    TUNING_CANDIDATES = (("direct", 16), ("direct", 32), ("direct", 64), ("tma", 16),
                         ("tma", 32))

    def fc2d_tuning(self):
        """(form "direct" or "tma", columns per block, {(form, columns): microseconds
        per extension step at plan time}) of the 4096-point column passes."""
        choice = np.zeros(2, np.int32)
        us = np.zeros(5, np.float32)
        _check(_lib.fc2d_tuning(self.handle, choice.ctypes.data, us.ctypes.data))
        return (("direct", "tma")[int(choice[1])], int(choice[0]),
                {c: float(v) for c, v in zip(self.TUNING_CANDIDATES, us)})

    def fc2d_tuning_set(self, columns_per_block, form="direct"):
        choice = np.array([columns_per_block, {"direct": 0, "tma": 1}[form]], np.int32)
        _check(_lib.fc2d_tuning_set(self.handle, choice.ctypes.data))

    def fc2d_profile(self, enable=True):
        _check(_lib.fc2d_profile(self.handle, 1 if enable else 0))

    def fc2d_profile_read(self, max_kernels=64):
        """{kernel name: (launches, total ms)} since the last read (the read clears)."""
        n = ct.c_int()
        names = ct.create_string_buffer(64 * max_kernels)
        launches = np.zeros(max_kernels, np.int64)
        ms = np.zeros(max_kernels)
        _check(_lib.fc2d_profile_read(self.handle, max_kernels, names, launches.ctypes.data,
                                      ms.ctypes.data, ct.byref(n)))
        raw = names.raw
        k = min(n.value, max_kernels)
        return {raw[64 * i:64 * i + 64].split(b"\0")[0].decode(): (int(launches[i]), float(ms[i]))
                for i in range(k)}

    def fc2d_sync_status(self, stream=None):
        _check(_lib.fc2d_sync_status(self.handle, _stream(stream)))

    def fc2d_wait_selftest(self, polls, stream=None):
        _check(_lib.fc2d_wait_selftest(self.handle, int(polls), _stream(stream)))

    def fc2d_destroy(self):
        if self.handle:
            _lib.fc2d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.fc2d_destroy()
        except Exception:
            pass


def fc2d_plan(boundary, grid, params=None, precision=FC2D_FP64) -> Plan:
    return Plan(boundary, grid, params, precision)


class Group:
    """A plan group: the extension + DFT of several domains as one CUDA graph, each plan
    on its own branch (fc2d_group_create).  Keeps references to its plans."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ct.c_void_p * len(self.plans))(*[pl.handle for pl in self.plans])
        h = ct.c_void_p()
        _check(_lib.fc2d_group_create(arr, len(self.plans), ct.byref(h)))
        self.handle = h

    def fc2d_group_extend_coeffs(self, n_f, f_grid, f_bdry, fhat, stream=None):
        """n_f: per plan; f_grid, fhat: per plan device tensors; f_bdry: per plan tensors
        or None entries (interior data only), or None."""
        n = len(self.plans)
        nf = (ct.c_int * n)(*n_f)
        fg = (ct.c_void_p * n)(*[_ptr(x) for x in f_grid])
        fh = (ct.c_void_p * n)(*[_ptr(x) for x in fhat])
        fb = None if f_bdry is None else (ct.c_void_p * n)(*[_ptr(x) for x in f_bdry])
        _check(_lib.fc2d_group_extend_coeffs(self.handle, nf, fg, fb, fh, _stream(stream)))

    def fc2d_group_tuning(self):
        """(form kept: "persistent" or "branches", persistent kernel threads per CTA,
        {"queue256", "queue512", "branches", "persistent"}: microseconds per launch)."""
        ch = (ct.c_int32 * 2)()
        us = (ct.c_float * 4)()
        _check(_lib.fc2d_group_tuning(self.handle, ch, us))
        return ("persistent" if ch[0] else "branches", ch[1],
                dict(zip(("queue256", "queue512", "branches", "persistent"), us)))

    def fc2d_group_tuning_set(self, form=None, threads=256):
        """Fix the captured form ("persistent" or "branches") and the persistent kernel's
        threads per CTA for later captures; form None: tune again."""
        if form is None:
            _check(_lib.fc2d_group_tuning_set(self.handle, None))
        else:
            ch = (ct.c_int32 * 2)(1 if form == "persistent" else 0, threads)
            _check(_lib.fc2d_group_tuning_set(self.handle, ch))

    def fc2d_group_destroy(self):
        if self.handle:
            _lib.fc2d_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.fc2d_group_destroy()
        except Exception:
            pass


def fc2d_probe_fp64(out, blocks, iters, stream=None):
    """Launch the FP64 fused multiply-add probe; returns the flops it performs."""
    flops = ct.c_double()
    _check(_lib.fc2d_probe_fp64(_ptr(out), blocks, iters, ct.byref(flops), _stream(stream)))
    return flops.value


def fc2d_group_create(plans) -> Group:
    return Group(plans)
