"""Build and run tests/host_plan_harness.cpp: the library's host plan on the CPU."""
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_plan_harness.cpp")
EXE = os.path.join(ROOT, "_build", "host_plan_harness")


def build():
    deps = [SRC] + [os.path.join(ROOT, "paper_2010_03901_gb300", "csrc", f)
                    for f in ("plan.cpp", "plan_internal.h", "dd.h", "wave_band.cpp",
                              "wave_band.h")]
    if os.path.exists(EXE) and all(os.path.getmtime(d) < os.path.getmtime(EXE) for d in deps):
        return EXE
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    cuda = "/usr/local/cuda"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + cuda + "/include",
           "-I" + os.path.join(ROOT, "include"), SRC, "-o", EXE, "-L" + cuda + "/lib64",
           "-lcudart", "-Wl,-rpath," + cuda + "/lib64"]
    subprocess.run(cmd, check=True, capture_output=True)
    return EXE


def run(w, n_c=None, squares=False):
    """The plan's host tables; with n_c also the Fourier Forwarding band (wb_*), and with
    squares the band of the small-square procedure and its squares (sq_*)."""
    exe = build()
    cx, sx, cy, sy = w.boundary.arrays()
    g, p = w.grid, w.params
    args = [str(len(cx))] + [repr(float(v)) for arr in (cx, sx, cy, sy) for v in arr]
    args += [repr(float(g.a0)), repr(float(g.b0)), repr(float(g.h)), str(g.nx), str(g.ny)]
    args += [str(v) for v in (p.d, p.C, p.Z, p.n_os, p.n_r, p.M, p.B, p.m_F)] + [repr(float(p.k1))]
    if n_c is not None:
        args.append(str(int(n_c)))
        if squares:
            args.append("1")
    out = subprocess.run([exe] + args, check=True, capture_output=True).stdout
    res = {}
    pos = out.index(b"\n")
    head = out[:pos].decode().split(maxsplit=2)
    res["status"] = int(head[1])
    res["error"] = head[2] if len(head) > 2 else ""
    pos += 1
    types = {8: np.float64, 4: np.int32}
    while pos < len(out):
        end = out.index(b"\n", pos)
        if out[pos:end].startswith((b"wave_status", b"squares_status")):
            head = out[pos:end].decode().split(maxsplit=2)
            key = head[0].split("_")[0]
            res[key + "_status"] = int(head[1])
            res[key + "_error"] = head[2] if len(head) > 2 else ""
            pos = end + 1
            continue
        name, n, sz = out[pos:end].decode().split()
        n, sz = int(n), int(sz)
        dt = types[sz]
        if name in ("row_iv_off", "row_iv", "strip_lin", "gidx", "gidx_c", "row_iv_coff",
                    "gidx_i", "interior_ok") or (name.startswith(("wb_", "sq_")) and sz == 4):
            dt = np.uint32 if name.endswith("_col") else np.int32
        arr = np.frombuffer(out[end + 1:end + 1 + n * sz], dtype=dt)
        res[name] = arr
        pos = end + 1 + n * sz + 1
    return res


def partition(cnt, cap, n_cta):
    """The plan's ownership ranges (partition_owners) for points-per-normal counts."""
    exe = build()
    inp = f"{cap} {n_cta} {len(cnt)} " + " ".join(str(int(v)) for v in cnt)
    out = subprocess.run([exe, "partition"], input=inp.encode(), check=True,
                         capture_output=True).stdout
    return np.array([int(t) for t in out.split()], dtype=np.int64)
