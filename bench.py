#!/usr/bin/env python
"""Benchmark: 2D-FC extension + 2D DFT throughput (grid points per second) on the kite
domain x = cos t + 0.65 cos 2t - 0.65, y = 1.5 sin t at 4096^2 with 8192 normals.

One step = the whole hot path for one function: matching values, blending, strip
interpolation, fused extension + row DFT, column DFT (fc2d_extend_coeffs).  The headline
is the mixed-precision form; the FP64 form is timed beside it, and both spectra are
compared with the FP64 oracle's.  The Poisson solve on the star workload at 1024^2 is
reported as a second line item.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...     # the FP64 CPU oracle as the reference arm

Prints ONE JSON line (rank 0).  With --gpus N > 1 (launched by torch.distributed.run)
each rank runs an independent replica of the workload on its own GPU: the path has no
exchange step, so there is no collective beyond the timing barrier and max-reduce.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "kite4096"
METRIC = "2D-FC extend+FFT grid-points/sec at 4096^2"
UNIT = "grid-points/s"
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal; 152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz)
# FP32 issue rate: 152 SMs x 128 FP32 lanes x 2.07 GHz (nominal maximum SM clock)
FP32_PEAK_GINSTR = 152 * 128 * 2.07
# FP32 instructions per (point, node) term of the double-float double-layer sums
# (k_dlp): two coordinate differences 22, the term 82, the accumulation 11
DLP_INSTR_PER_TERM = 115

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel scope
# on this workload, from one ncu capture of the current kernels (cold cache, serialised
# launches; a scope with two kernels sums both).  A kernel changed after its capture
# has no entry, and the roofline then reports traffic null.
ROT = 3   # rotating input/output buffers of the timed steps
# kernels launched inside one profiled scope where it is more than one: the FP32
# 4096-point column DFT runs in two passes (k_cols4k_a, k_cols4k_b)
KERNELS_PER_SCOPE = {("mixed", "fft_cols", 4096): 2}

MEASURED_TRAFFIC = {
    ("mixed", "fft_rows_fused"): 70898688 + 8000768,
    ("mixed", "gather_blend_interp_tc"): 34114048 + 0,
    ("mixed", "fft_cols"): (67674624 + 7534592) + (67655168 + 6790400),
    ("fp64", "fft_rows_fused"): 72354816 + 72103424,
    ("fp64", "fft_cols"): 141867520 + 92843264,
    ("fp64", "gather_blend"): 9670144 + 9472,
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- #
# clocks during the timed region
# --------------------------------------------------------------------------- #
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- #
# the oracle (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------- #
def oracle_setup(w):
    from oracle import fc2d as OF
    from oracle import geometry as OG
    from oracle.fc_matrices import load_fc_matrices
    geo = OG.build_geometry(w)
    st = OF.matching_stencils(geo)
    return geo, st, load_fc_matrices()


def oracle_step(w, geo, st, mats, f):
    from oracle import fc2d as OF
    fg = W.grid_values(w, f)
    fb = OF.boundary_values(geo, f)
    t = time.perf_counter()
    out = OF.coefficients(OF.extension(geo, mats, fg, fb, st))
    return out, time.perf_counter() - t


def bench_functions(w, n):
    return [W.gaussian_sum(w.boundary, 16, 3 + k) for k in range(n)]


def cpu_info():
    """nproc, the CPU model and the BLAS thread count of this host."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            txt = fh.read()
        for key in ("model name", "Model", "Hardware", "CPU part"):
            for ln in txt.splitlines():
                if ln.lower().startswith(key.lower()) and ":" in ln:
                    model = f"{key}: {ln.split(':', 1)[1].strip()}"
                    break
            if model:
                break
    except OSError:
        pass
    blas = None
    try:
        from threadpoolctl import threadpool_info
        blas = [{"api": d.get("internal_api"), "threads": d.get("num_threads")}
                for d in threadpool_info()]
    except Exception:
        blas = "threadpoolctl unavailable"
    return {"nproc": os.cpu_count(), "affinity_cores": len(os.sched_getaffinity(0)),
            "model": model or platform.machine(), "blas": blas}


_CPU_STATE = {}


def _cpu_worker_init(path, name):
    """Spawned worker: one core's oracle, single-threaded (the parent pins its BLAS and
    FFT thread counts to 1 in the environment before spawning)."""
    import pickle
    with open(path, "rb") as fh:
        _CPU_STATE["setup"] = pickle.load(fh)
    _CPU_STATE["w"] = W.workload(name)


def _cpu_worker_run(args):
    """Functions index0, index0 + stride, ... until `budget` seconds of work."""
    index0, stride, budget = args
    geo, st, mats = _CPU_STATE["setup"]
    w = _CPU_STATE["w"]
    fs = bench_functions(w, 64)
    total, n, k = 0.0, 0, index0
    while total < budget:
        _, dt = oracle_step(w, geo, st, mats, fs[k % len(fs)])
        total += dt
        n += 1
        k += stride
    return n


def cpu_baseline(w, budget_s=15.0, all_budget_s=8.0):
    """The oracle as it stands on the full workload grid: extension + DFT per function
    (plan excluded, as on the GPU).  Single core: this process pinned to one core
    (sched_setaffinity, so every BLAS or FFT thread shares it), functions until the
    budget is used.  All cores: one spawned process per allowed core (BLAS and FFT
    threads 1 each), every process running functions for all_budget_s; the points of
    all of them over the wall time of the whole batch."""
    import multiprocessing as mp
    import pickle
    import tempfile
    geo, st, mats = oracle_setup(w)
    npts = w.grid.nx * w.grid.ny
    allowed = os.sched_getaffinity(0)
    total, n, first = 0.0, 0, None
    os.sched_setaffinity(0, {min(allowed)})
    try:
        for f in bench_functions(w, 64):
            out, dt = oracle_step(w, geo, st, mats, f)
            if first is None:
                first = out
            total += dt
            n += 1
            if total >= budget_s:
                break
    finally:
        os.sched_setaffinity(0, allowed)
    ncores = len(allowed)
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    all_cores = None
    with tempfile.NamedTemporaryFile(suffix=".pkl", delete=False) as tmp:
        pickle.dump((geo, st, mats), tmp, protocol=pickle.HIGHEST_PROTOCOL)
        path = tmp.name
    try:
        for k in env_keys:
            os.environ[k] = "1"
        ctx = mp.get_context("spawn")  # the GPU context of this process must not fork
        with ctx.Pool(ncores, initializer=_cpu_worker_init, initargs=(path, w.name)) as pool:
            limit = 600.0  # a worker that cannot start must not hang the benchmark
            pool.map_async(_cpu_worker_run, [(i, ncores, 0.0) for i in range(ncores)]).get(limit)
            t0 = time.perf_counter()
            counts = pool.map_async(_cpu_worker_run,
                                    [(i, ncores, all_budget_s) for i in range(ncores)]).get(limit)
            wall = time.perf_counter() - t0
        all_cores = {"value": sum(counts) * npts / wall, "unit": UNIT, "cores": ncores,
                     "sample": f"{sum(counts)} functions on {ncores} spawned single-threaded "
                               f"processes, {wall:.1f} s wall"}
    except Exception as e:  # the single-core figure stands on its own
        all_cores = {"unavailable": f"{type(e).__name__}: {e}"}
    finally:
        os.unlink(path)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": n * npts / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} function(s) of the {w.name} workload, full grid, plan excluded; "
                      f"{total:.1f} s of CPU on one pinned core",
            "all_cores": all_cores, "host": cpu_info()}, first


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # step = one oracle extension + DFT of the kite; the grid is the largest of
    # 4096^2, 2048^2, 1024^2 that keeps the whole run near two minutes
    est4096 = 2.5  # seconds per step on one core at 4096^2 (measured on the dev host)
    n_steps = args.steps + args.warmup
    name = "kite4096"
    for cand, scale in (("kite4096", 1.0), ("kite2048", 0.25)):
        name = cand
        if n_steps * est4096 * scale <= 120:
            break
    else:
        name = "kite1024"
    w = W.workload(name)
    geo, st, mats = oracle_setup(w)
    f = bench_functions(w, 1)[0]
    for _ in range(args.warmup):
        oracle_step(w, geo, st, mats, f)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_step(w, geo, st, mats, f)[1]
    npts = w.grid.nx * w.grid.ny
    value = args.steps * npts / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_grid": f"{w.grid.nx}x{w.grid.ny}",
                       "domain": "kite a=0.65 b=1.5", "normals": w.params.B,
                       "functions": "sum of 16 Gaussians, seed 3"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{w.name}: one function per step, plan excluded"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# the GPU arm
# --------------------------------------------------------------------------- #
def algorithmic(plan, w, fp64):
    """Algorithmic bytes and flops per launch of each kernel scope (one function)."""
    g = w.grid
    nx, ny = g.nx, g.ny
    nh = nx // 2
    esz = 8 if fp64 else 4
    csz = 2 * esz
    spec = ny * (nh + 1) * csz
    B = w.params.B
    Cr = w.params.C * w.params.n_r
    M = w.params.M
    fft_rows_flops = ny * (5.0 * nh * math.log2(nh) + 10.0 * (nh + 1))
    fft_cols_flops = (nh + 1) * 5.0 * ny * math.log2(ny)
    gather = {"bytes": B * ((M - 1) * M * 12 + (w.params.d - 1) * M * 8 + (Cr + 1) * esz),
              "flops": B * 2.0 * ((M - 1) * M + (w.params.d - 1) * M + Cr * w.params.d)}
    interp = {"bytes": plan.n_strip * (16 + esz), "flops": plan.n_strip * 2.0 * (M * M + M)}
    return {
        "fft_rows_fused": {"bytes": 8 * plan.n_inside + (esz + 4) * plan.n_strip + spec,
                           "flops": fft_rows_flops},
        # blend + interpolation in one kernel: the gather's taps, the weights (2M x 4 B),
        # the grouped index and packed nodes (8 B) and the value (4 B) of each strip point
        "gather_blend_interp_tc": {
            "bytes": gather["bytes"] - B * (Cr + 1) * esz + plan.n_strip * (2 * M * 4 + 8 + 4),
            "flops": gather["flops"] + interp["flops"]},
        "fft_cols": {"bytes": 2 * spec, "flops": fft_cols_flops},
        "interp": interp,
        "gather_blend": gather,
    }


def max_over_ranks(x, world, dev):
    """The largest value of x over all ranks (the slowest replica's time).  Works on any
    process-group backend: NCCL with a CUDA device, gloo with the CPU."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, points_per_step, ms):
    """Whole-job points/s: every rank processes `steps` grids of `points_per_step` points
    (replicas, weak scaling), divided by the slowest rank's time `ms`."""
    return world * steps * points_per_step / (ms / 1e3)


def measure(fc2d, torch, w, precision, K, warmup, world, dev, fg_h, fb_h, sample_clocks):
    """Time K steps of fc2d_extend_coeffs (one function) in one precision; per-kernel
    CUDA-event profile over the same timed region; e2e with host buffers."""
    g, p = w.grid, w.params
    fp64 = precision == "fp64"
    t0 = time.perf_counter()
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1),
                          precision=fc2d.FC2D_FP64 if fp64 else fc2d.FC2D_MIXED)
    plan_s = time.perf_counter() - t0
    # inputs larger than L2: ROT copies of f on the whole grid (FP64, 134 MB each at
    # 4096^2, above the 129 MB of L2) and ROT spectra, used in turn, so that no step finds
    # another step's input or output in L2
    fgs = [fg_h.to(dev) for _ in range(ROT)]
    fb = fb_h.to(dev)
    fg = fgs[0]
    cdt = torch.float64 if fp64 else torch.float32
    fhats = [torch.zeros((g.ny, g.nx // 2 + 1, 2), dtype=cdt, device=dev) for _ in range(ROT)]
    fhat = fhats[0]
    # for the flushed variant: a read-only pass over 256 MB (> 129 MB of L2) before each
    # step, which evicts the previous step's data without leaving dirty lines behind
    flush = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    flush_out = torch.empty(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for k in range(warmup):
        plan.fc2d_extend_coeffs(1, fgs[k % ROT], fb, fhats[k % ROT], stream)
    plan.fc2d_sync_status(stream)
    sampler = ClockSampler(dev.index) if sample_clocks else None

    def timed_region(profile=False, flushed=False):
        """K steps of fc2d_extend_coeffs.  Default: back to back between two events,
        each step on the next of the ROT input/output buffers.  flushed: the L2 flushed
        before each step, outside per-step events.  profile: the library also records
        CUDA events around each of its kernels."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        if profile:
            plan.fc2d_profile(True)
            plan.fc2d_profile_read()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            if flushed:
                torch.sum(flush, dim=0, out=flush_out[0])
            if flushed or k == 0:
                starts[k].record(stream)
            plan.fc2d_extend_coeffs(1, fgs[k % ROT], fb, fhats[k % ROT], stream)
            if flushed or k == K - 1:
                ends[k].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        prof = None
        if profile:
            plan.fc2d_profile(False)
            prof = plan.fc2d_profile_read()
        plan.fc2d_sync_status(stream)
        if flushed:
            return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), prof
        return starts[0].elapsed_time(ends[K - 1]), prof

    # the headline: K steps back to back, nothing between the library's kernels
    # (per-kernel events would stop each kernel's launch from overlapping the previous
    # one's tail)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    wall0 = time.perf_counter()
    ms_raw, _ = timed_region()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ms_raw, world, dev)
    # the same K steps with the L2 flushed before each step (outside the events)
    ms_fl = max_over_ranks(timed_region(flushed=True)[0], world, dev)
    # the per-kernel profile (roofline, launch count): the same K steps again with the
    # library's CUDA events around each kernel
    ms_prof_raw, prof = timed_region(profile=True)
    ms_prof = max_over_ranks(ms_prof_raw, world, dev)
    npts = g.nx * g.ny
    value = replica_throughput(world, K, npts, ms)
    # end to end through the public API with host buffers: every step copies its
    # inputs from pinned host memory, calls the library and reads its spectrum back to
    # pinned host memory.  Steps are pipelined as a user streaming functions would:
    # copies in on one stream, compute on another, copies out on a third, with two
    # device buffers of each kind (the plan's workspace is used by one compute stream
    # only).  The headline form passes f at the domain's grid points only
    # (fc2d_extend_coeffs_compact, the method's data); the full-grid form
    # (fc2d_extend_coeffs) is timed beside it.
    lin = torch.from_numpy(plan.fc2d_inside_points())
    fin_h = fg_h.reshape(-1)[lin].contiguous().pin_memory()

    def e2e(compact):
        Ke = min(K, 30)
        src_h = fin_h if compact else fg_h
        fhat_h = [torch.empty(fhat.shape, dtype=cdt).pin_memory() for _ in range(2)]
        fg_d = [torch.empty(src_h.shape, dtype=src_h.dtype, device=dev) for _ in range(2)]
        fb_d = [torch.empty_like(fb) for _ in range(2)]
        fh_d = [torch.empty_like(fhat) for _ in range(2)]
        s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev = lambda: torch.cuda.Event()
        in_done = [ev(), ev()]
        cmp_done = [ev(), ev()]
        out_done = [ev(), ev()]
        call = plan.fc2d_extend_coeffs_compact if compact else plan.fc2d_extend_coeffs

        def step(k):
            b = k % 2
            with torch.cuda.stream(s_in):
                s_in.wait_event(cmp_done[b])      # compute k-2 has read these inputs
                fg_d[b].copy_(src_h, non_blocking=True)
                fb_d[b].copy_(fb_h, non_blocking=True)
                in_done[b].record(s_in)
            s_cmp.wait_event(in_done[b])
            s_cmp.wait_event(out_done[b])         # copy-out k-2 has read this spectrum
            call(1, fg_d[b], fb_d[b], fh_d[b], s_cmp)
            cmp_done[b].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(cmp_done[b])
                fhat_h[b].copy_(fh_d[b], non_blocking=True)
                out_done[b].record(s_out)

        torch.cuda.synchronize()
        for k in range(2):
            step(k)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        for k in range(Ke):
            step(k)
        for b in range(2):
            s_out.wait_event(out_done[b])
        e1.record(s_out)
        torch.cuda.synchronize()
        plan.fc2d_sync_status(s_cmp)
        ms_step = max_over_ranks(e0.elapsed_time(e1) / Ke, world, dev)
        h2d = int(src_h.numel() * src_h.element_size() + fb_h.numel() * fb_h.element_size())
        return ms_step, h2d

    e2e_ms, e2e_h2d = e2e(True)
    e2e_full_ms, e2e_full_h2d = e2e(False)
    link = host_link(torch, dev, e2e_h2d, int(fhat.numel() * fhat.element_size()))
    # roofline of the dominant kernel
    hbm, src = peaks()
    alg = algorithmic(plan, w, fp64)
    dom = max(prof, key=lambda k: prof[k][1])
    launches, tot_ms = prof[dom]
    avg_s = tot_ms / launches / 1e3
    a = alg.get(dom, {"bytes": 0, "flops": 0})
    t_hbm = a["bytes"] / (hbm * 1e9)
    fp64_tf = fp64_rate(fc2d, torch, dev) if fp64 else FP64_PEAK_TFLOPS
    t_alu = a["flops"] / (fp64_tf * 1e12) if fp64 else 0.0
    if fp64 and t_alu > t_hbm:
        roof = {"bound": "alu", "achieved": a["flops"] / avg_s / 1e12, "peak": fp64_tf,
                "unit": "TFLOP/s", "peak_source": "measured FP64 FMA rate (fp64_peak)"}
    else:
        roof = {"bound": "hbm", "achieved": a["bytes"] / avg_s / 1e9, "peak": hbm,
                "unit": "GB/s", "peak_source": src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dom
    # the column passes' stored traffic is per form (direct or TMA-pipelined)
    tk = (precision, dom) + (("tma",) if dom == "fft_cols" and
                             plan.fc2d_tuning()[0] == "tma" else ())
    roof["traffic"] = MEASURED_TRAFFIC.get(tk)
    roof["traffic_source"] = ("stored: one ncu capture (dram__bytes_read.sum + "
                              "dram__bytes_write.sum, cold cache) of this kernel on this "
                              "workload, not measured in this run" if roof["traffic"] else
                              "no capture of the current kernel")
    kernels = {k: {"launches": v[0], "avg_us": 1e3 * v[1] / v[0],
                   "share": v[1] / sum(x[1] for x in prof.values())} for k, v in prof.items()}
    cform, cc, cc_us = plan.fc2d_tuning()
    return {"value": value, "ms_per_step": ms / K, "steps": K, "plan_s": plan_s,
            "tuning": {"cols4k_form": cform, "cols4k_columns_per_block": cc,
                       "candidates_us_per_step": {f"{f}{c}": v for (f, c), v in
                                                  cc_us.items()},
                       "how": "plan-time autotuner: the column passes' direct form at "
                              "16/32/64 columns and TMA-pipelined form at 16/32, each "
                              "timed inside the plan's own extension step (synthetic "
                              "input, 10 steps), fastest kept (same values)"},
            "l2_flushed": {"value": replica_throughput(world, K, npts, ms_fl),
                           "ms_per_step": ms_fl / K,
                           "note": "L2 flushed before each step (256 MB read, outside "
                                   "per-step events)"},
            "profiled_ms_per_step": ms_prof / K,
            "wall_s_timed": wall, "clocks": clocks, "roofline": roof, "kernels": kernels,
            "gpu_launches": sum(v[0] * KERNELS_PER_SCOPE.get((precision, k, g.ny), 1)
                                for k, v in prof.items()),
            "e2e": {"value": replica_throughput(world, 1, npts, e2e_ms), "unit": UNIT,
                    "api": "fc2d_extend_coeffs_compact (f at the domain's grid points)",
                    "pipeline": "copy-in, compute, copy-out on three streams, two buffers",
                    "h2d_bytes_per_step": e2e_h2d,
                    "d2h_bytes_per_step": int(fhat.numel() * fhat.element_size()),
                    "ms_per_step": e2e_ms, "host_link": link,
                    "full_grid": {"api": "fc2d_extend_coeffs (f on the whole grid)",
                                  "value": replica_throughput(world, 1, npts, e2e_full_ms),
                                  "h2d_bytes_per_step": e2e_full_h2d}},
            "fhat": fhat}


def host_link(torch, dev, h2d_bytes, d2h_bytes, reps=10):
    """The host link alone, with the e2e pipeline's byte counts: pinned-memory copies of
    h2d_bytes in and d2h_bytes out, each direction alone and both at once on two
    streams (GB/s per direction, CUDA events), and the step time those copies alone
    would take with both directions busy."""
    h_in = torch.empty(h2d_bytes // 8, dtype=torch.float64).pin_memory()
    h_out = torch.empty(d2h_bytes // 8, dtype=torch.float64).pin_memory()
    d_in = torch.empty(h_in.numel(), dtype=torch.float64, device=dev)
    d_out = torch.empty(h_out.numel(), dtype=torch.float64, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    cur = torch.cuda.current_stream(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        for _ in range(reps):
            fn()
        b.record(cur)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def both():
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    t_in = timed(lambda: d_in.copy_(h_in, non_blocking=True))
    t_out = timed(lambda: h_out.copy_(d_out, non_blocking=True))
    t_both = timed(both)
    return {"h2d_GBs": h2d_bytes / t_in / 1e6, "d2h_GBs": d2h_bytes / t_out / 1e6,
            "both_ms": t_both,
            "note": "the step's copies alone, both directions at once: the e2e floor"}


def poisson_star1024(fc2d, torch, dev, solves=3):
    """The star r = 1 + 0.3 cos 5 theta at 1024^2: Poisson with u = sin(2x) e^y (FP64)."""
    w = W.workload("star1024")
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(B=p.B, k1=p.k1))
    plan.fc2d_poisson_plan(0)
    xy = plan.fc2d_poisson_nodes()
    bxy = plan.fc2d_boundary_points()
    f, u = W.lap_u_manufactured, W.u_manufactured
    fg = torch.tensor(W.grid_values(w, f)[None], device=dev)
    fb = torch.tensor(f(bxy[:, 0], bxy[:, 1])[None], device=dev)
    gn = torch.tensor(u(xy[:, 0], xy[:, 1])[None], device=dev)
    out = torch.zeros_like(fg)
    plan.fc2d_poisson(1, fg, fb, gn, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(solves):
        plan.fc2d_poisson(1, fg, fb, gn, out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / solves
    plan.fc2d_profile(True)
    plan.fc2d_profile_read()
    plan.fc2d_poisson(1, fg, fb, gn, out)
    torch.cuda.synchronize()
    plan.fc2d_profile(False)
    prof = plan.fc2d_profile_read()
    X, Y = np.meshgrid(*w.grid.coords())
    ue = u(X, Y)
    got = out.cpu().numpy()[0]
    inside = got != 0
    err = float(np.abs(got - ue)[inside].max() / np.abs(ue[inside]).max())
    info = plan.fc2d_poisson_info()
    kms = {k: v[1] / v[0] for k, v in prof.items()}
    # the far-field sums: (inside points - near points) x N_b terms, FP32-issue bound
    terms = (plan.n_inside - info["n_near"]) * len(xy)
    ach = terms * DLP_INSTR_PER_TERM / (kms["dlp_far"] * 1e-3) / 1e9
    roof = {"bound": "alu", "kernel": "dlp_far (k_dlp<false>, N_b nodes)", "achieved": ach,
            "peak": FP32_PEAK_GINSTR, "unit": "G FP32 instr/s", "frac": ach / FP32_PEAK_GINSTR,
            "terms": terms, "instr_per_term": DLP_INSTR_PER_TERM,
            "peak_source": "nominal: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    return {"workload": "star1024 Poisson, u = sin(2x) e^y", "ms_per_solve": 1e3 * dt,
            "value": g.nx * g.ny / dt, "unit": UNIT, "max_rel_err_vs_exact": err,
            "gmres": info, "kernels_ms": kms, "roofline": roof}


def poisson_kite_oscillatory(fc2d, torch, dev, h=1.25e-3, solves=3):
    """Example 4.3 (Table 4) at its finest step: f = -sin(40 pi x) sin(40 pi y) on the
    kite x = cos t + 0.35 cos 2t - 0.35, y = 0.7 sin t, d = 10, M = M_P = 13, FP64;
    relative errors against u = sin(40 pi x) sin(40 pi y)/(3200 pi^2) over the grid
    points inside at a distance > 0.2 from the curve (the paper prints 5.8e-12 l_inf and
    1.6e-12 l_2 at this h)."""
    b = W.kite(0.35, 0.7)
    px, py = b.polygon(20000)
    g = W.fit_grid_smooth(px.min(), px.max(), py.min(), py.max(), h)
    B = int(round(2 * np.pi / h))
    plan = fc2d.fc2d_plan(b.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=10, M=13, B=B, k1=h))
    plan.fc2d_poisson_plan(0)
    xy = plan.fc2d_poisson_nodes()
    bxy = plan.fc2d_boundary_points()
    a = 40 * np.pi
    u = lambda x, y: np.sin(a * x) * np.sin(a * y) / (2 * a * a)
    f = lambda x, y: -np.sin(a * x) * np.sin(a * y)
    xs, ys = g.coords()
    X, Y = np.meshgrid(xs, ys)
    fg = torch.tensor(f(X, Y)[None], device=dev)
    fb = torch.tensor(f(bxy[:, 0], bxy[:, 1])[None], device=dev)
    gn = torch.tensor(u(xy[:, 0], xy[:, 1])[None], device=dev)
    out = torch.zeros_like(fg)
    plan.fc2d_poisson(1, fg, fb, gn, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(solves):
        plan.fc2d_poisson(1, fg, fb, gn, out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / solves
    far = W.far_inside(b, xs, ys, 0.2)
    ue = u(X, Y)[far]
    e = out.cpu().numpy()[0][far] - ue
    return {"workload": f"paper kite, f = -sin(40 pi x) sin(40 pi y), d = 10, h = {h}, "
                        f"{g.nx}x{g.ny}",
            "ms_per_solve": 1e3 * dt, "value": g.nx * g.ny / dt, "unit": UNIT,
            "rel_linf_far": float(np.abs(e).max() / np.abs(ue).max()),
            "rel_l2_far": float(np.sqrt(np.mean(e ** 2) / np.mean(ue ** 2))),
            "paper_rel_linf": 5.8e-12, "paper_rel_l2": 1.6e-12,
            "gmres": plan.fc2d_poisson_info()}


def ff_interior_kite2048(fc2d, torch, dev, steps=20):
    """One Fourier Forwarding large step, the interior propagator U_FC (Section 4.2):
    both extensions, both DFTs, the modal advance, both inverse DFTs.  The kite at 2048^2
    with d = 4 (the paper's FF order), c = 1, Delta T = n_c h with n_c = 8; u = 32
    Gaussians of width 0.05 centred at least 0.3 inside the curve (seed 5), u_t = 0;
    FP64.  Calls back to back on the launching stream between two events."""
    w = W.workload("kite2048", d=4, M=7)
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    xy = plan.fc2d_boundary_points()
    f0 = W.gaussian_sum(w.boundary, 32, 5, wmin=0.05, wmax=0.05, margin=0.3)
    u0 = torch.tensor(W.grid_values(w, f0)[None], device=dev)
    ub = torch.tensor(f0(xy[:, 0], xy[:, 1])[None], device=dev)
    ut0, utb = torch.zeros_like(u0), torch.zeros_like(ub)
    u1, ut1 = torch.empty_like(u0), torch.empty_like(u0)
    dT = 8 * g.h
    stream = torch.cuda.current_stream()
    for _ in range(3):
        plan.fc2d_wave_interior(1, 1.0, dT, u0, ub, ut0, utb, u1, ut1, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        plan.fc2d_wave_interior(1, 1.0, dT, u0, ub, ut0, utb, u1, ut1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plan.fc2d_profile(True)
    plan.fc2d_profile_read()
    plan.fc2d_wave_interior(1, 1.0, dT, u0, ub, ut0, utb, u1, ut1, stream)
    torch.cuda.synchronize()
    plan.fc2d_profile(False)
    prof = plan.fc2d_profile_read()
    plan.fc2d_sync_status(stream)
    kms = {k: v[1] / v[0] for k, v in prof.items()}
    # k_wave_cols: per spectrum (u and u_t) a forward and an inverse column DFT of ny
    # points on nx/2 + 1 columns, 5 ny log2(ny) flops each (the modal advance not counted)
    flops = 4 * (g.nx // 2 + 1) * 5 * g.ny * np.log2(g.ny)
    ach = flops / (kms["wave_cols"] * 1e-3) / 1e12
    return {"workload": f"kite 2048^2 (a=0.65, b=1.5), d = 4, c = 1, Delta T = 8 h = {dT:.4g}, "
                        "u = 32 Gaussians (w = 0.05, centres >= 0.3 inside), u_t = 0",
            "ms_per_large_step": ms, "large_steps_per_s": 1e3 / ms,
            "value": g.nx * g.ny / (ms * 1e-3), "unit": UNIT, "kernels_ms": kms,
            "roofline": {"bound": "alu", "kernel": "wave_cols (k_wave_cols_p2)", "achieved": ach,
                         "peak": fp64_rate(fc2d, torch, dev), "unit": "TFLOP/s",
                         "frac": ach / fp64_rate(fc2d, torch, dev),
                         "peak_source": "measured FP64 FMA rate (fp64_peak)",
                         "flops": "4 column DFTs x 5 N log2 N, modal advance not counted"}}


def fp64_peak(fc2d, torch, dev, iters=1 << 16):
    """Measured FP64 rate (TFLOP/s): the library's fused multiply-add probe on
    8 x 152 blocks of 256 threads, best of 3 timed launches (CUDA events), with the SM
    clock sampled during them (a rate at another clock scales with it)."""
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * n_sm
    out = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    fc2d.fc2d_probe_fp64(out, blocks, 1024, stream)
    clk = ClockSampler(dev.index or 0)
    clk.start()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = fc2d.fc2d_probe_fp64(out, blocks, iters, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return {"tflops": best, "clocks": clk.stop(), "how": f"{blocks} blocks x 256 threads x 8 "
            f"independent FMA chains x {iters} steps, best of 3 (CUDA events)"}


_FP64_RATE = {}


def fp64_rate(fc2d, torch, dev):
    """The measured FP64 rate (TFLOP/s, fp64_peak), once per process."""
    if "tflops" not in _FP64_RATE:
        _FP64_RATE.update(fp64_peak(fc2d, torch, dev))
    return _FP64_RATE["tflops"]


def _disk_eigenmode_error(fc2d, torch, dev, h=0.005, n_c=8, T_target=2.0):
    """Fourier Forwarding of the disk eigenmode J_2(j r) cos(2 phi) cos(j t),
    j = j_{2,3} (zero Dirichlet data), to t ~ 2: max error on the grid points inside."""
    from scipy.special import jn_zeros, jv
    j = float(jn_zeros(2, 3)[-1])
    B = int(round(2 * math.pi / h / 8)) * 8
    g0 = W.fit_grid_smooth(-1.0, 1.0, -1.0, 1.0, h)
    g = W.Grid(a0=g0.a0 - 0.31 * h, b0=g0.b0 - 0.17 * h, h=h, nx=g0.nx, ny=g0.ny)
    plan = fc2d.fc2d_plan(W.disk().arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=B, k1=h))
    x, y = g.coords()
    X, Y = np.meshgrid(x, y)
    mode = lambda t: jv(2, j * np.hypot(X, Y)) * np.cos(2 * np.arctan2(Y, X)) * np.cos(j * t)
    n_large = int(round(T_target / (n_c * h)))
    T = n_large * n_c * h
    u = torch.tensor(mode(0.0)[None], device=dev)
    ut = torch.zeros_like(u)
    plan.fc2d_forward_wave(1, 1.0, n_c, n_large, u, ut)
    plan.fc2d_sync_status()
    got = u.cpu().numpy()[0]
    inside = X * X + Y * Y < 1.0
    err = float(np.abs(got - mode(T))[inside & (got != 0)].max())
    return {"grid": f"{g.nx}x{g.ny}", "h": h, "n_c": n_c, "t": T, "small_steps": n_large * 8 * n_c,
            "max_abs_error": err}


def ff_solve_kite2048(fc2d, torch, dev, n_large=2, mode=1, extras=True):
    """The whole Fourier Forwarding solve (Section 4.2, eq. (4.9); fc2d_forward_wave): the
    kite at 2048^2, d = 4, c = 1, n_c = 8 (Delta T = 8 h, 64 small steps of CFL 0.125
    per large step), zero Dirichlet data, 32 initial conditions in one call (a Gaussian of
    width 0.05 each, centres at least 0.35 inside the curve, seeds 50..81, u_t = 0), FP64,
    with the paper's small-square interface procedure (interface mode 1).  One call of
    n_large large steps is timed between two events on the launching stream after a
    warm-up call (the band and scratch are built there); the per-kernel times come from a
    second, profiled call.  Beside it: the measured FP64 rate, the error of the same
    solver against the exact Dirichlet eigenmode (2, 3) of the unit disk at t ~ 2, and the
    same solve with the full inverse DFT at every small step (mode 0) and with the
    squares evaluated in double-float arithmetic (mode 2; there the dominant kernel's
    "TFLOP/s" counts the FP64-equivalent DFT flops it replaces)."""
    squares, double_float = mode >= 1, mode == 2
    w = W.workload("kite2048", d=4, M=7)
    g, p = w.grid, w.params
    n_c, n_f, c = 8, 32, 1.0
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    fs = [W.gaussian_sum(w.boundary, 1, 50 + k, wmin=0.05, wmax=0.05, margin=0.35)
          for k in range(n_f)]
    U0 = torch.tensor(np.stack([W.grid_values(w, f) for f in fs]), device=dev)
    u, ut = torch.empty_like(U0), torch.empty_like(U0)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    u.copy_(U0)
    ut.zero_()
    plan.fc2d_forward_wave(n_f, c, n_c, 1, u, ut, None, None, stream, squares=squares,
                           double_float=double_float)
    torch.cuda.synchronize()
    first_call_s = time.time() - t0
    u.copy_(U0)
    ut.zero_()
    clk = ClockSampler(dev.index or 0)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plan.fc2d_forward_wave(n_f, c, n_c, n_large, u, ut, None, None, stream, squares=squares,
                           double_float=double_float)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    plan.fc2d_sync_status(stream)
    got = u.cpu().numpy()
    finite = bool(np.isfinite(got).all())
    amp = float(np.abs(got).max())
    # per-kernel times (a second call with events around each kernel)
    u.copy_(U0)
    ut.zero_()
    plan.fc2d_profile(True)
    plan.fc2d_profile_read()
    plan.fc2d_forward_wave(n_f, c, n_c, n_large, u, ut, None, None, stream, squares=squares,
                           double_float=double_float)
    torch.cuda.synchronize()
    plan.fc2d_profile(False)
    prof = plan.fc2d_profile_read()
    counts = plan.fc2d_wave_band_info(n_c, squares=squares)
    S = 8 * n_c
    small = n_large * S
    peak = (dict(_FP64_RATE) if "tflops" in _FP64_RATE else None) if extras else None
    if extras and peak is None:
        fp64_rate(fc2d, torch, dev)
        peak = dict(_FP64_RATE)
    kms = {k: {"launches": v[0], "ms_per_launch": v[1] / v[0], "ms_total": v[1]}
           for k, v in prof.items()}
    # dominant kernel, FLOPs of one launch for n_f functions (5 N log2 N per length-N
    # complex DFT): the modal advance + inverse column DFT (k_ff_cols) or the inverse
    # rows of the full U_FC; with squares the per-small-step square inversion (k_sq_eval:
    # per square and function pair a 64 x 64 complex DFT, 2 x 64 x 5 x 64 x 6)
    nh = g.nx // 2
    flops = {"ff_cols": n_f * (nh + 1) * 5.0 * g.ny * math.log2(g.ny),
             "inverse_rows": n_f * g.ny * (5.0 * nh * math.log2(nh) + 10.0 * (nh + 1)),
             "sq_eval": counts[4] * ((n_f + 1) // 2) * 2 * 64 * 5.0 * 64 * 6}
    top = max(flops, key=lambda k: kms.get(k, {}).get("ms_total", 0.0))
    ach = flops[top] / (kms[top]["ms_per_launch"] * 1e-3) / 1e12
    if not extras:
        return {"ms_per_large_step": ms / n_large, "ms_per_small_step": ms / small,
                "small_steps_per_s": small / (ms * 1e-3), "finite": finite,
                "max_abs_u_end": amp, "squares": counts[4], "kernels": kms,
                "band": {"unknowns": counts[0], "interface": counts[2]}, "clocks": clocks,
                "top_kernel": top, "top_tflops": ach}
    eig = _disk_eigenmode_error(fc2d, torch, dev)
    return {"workload": f"kite 2048^2 (a=0.65, b=1.5), d = 4, c = 1, n_c = 8 (Delta T = 8 h), "
                        f"zero Dirichlet data, {n_f} initial conditions (one Gaussian each, "
                        "w = 0.05, centres >= 0.35 inside, seeds 50..81), u_t = 0, FP64; "
                        "interface values by the small-square procedure (interface mode 1)",
            "n_f": n_f, "large_steps": n_large, "small_steps": small,
            "ms": ms, "ms_per_large_step": ms / n_large, "ms_per_small_step": ms / small,
            "small_steps_per_s": small / (ms * 1e-3),
            "function_small_steps_per_s": n_f * small / (ms * 1e-3),
            "value": n_f * g.nx * g.ny * small / (ms * 1e-3), "unit": "grid-point small steps/s",
            "band": {"unknowns": counts[0], "slaved": counts[1], "interface": counts[2],
                     "near": counts[3]},
            "first_call_s": first_call_s, "finite": finite, "max_abs_u_end": amp,
            "clocks": clocks, "kernels": kms, "gpu_launches_per_call": sum(v[0] for v in prof.values()),
            "roofline": {"bound": "alu", "kernel": top, "achieved": ach, "peak": peak["tflops"],
                         "unit": "TFLOP/s", "frac": ach / peak["tflops"],
                         "peak_source": "measured FP64 FMA rate (fp64_peak)",
                         "flops": "5 N log2 N per length-N complex DFT of the launch"},
            "fp64_peak": peak, "disk_eigenmode": eig,
            "parity": "tests/test_gpu_ff.py (element-wise against the oracle)",
            "full_inverse_dft": ff_solve_kite2048(fc2d, torch, dev, n_large, mode=0,
                                                  extras=False),
            "small_squares_double_float": ff_solve_kite2048(fc2d, torch, dev, n_large, mode=2,
                                                            extras=False)}


def ff_scaling(fc2d, torch, dev, n_f=8, n_c=8):
    """Cost of a Fourier Forwarding small step against the grid size (Section 4.2: with
    the small-square procedure the interface values cost O(perimeter / h) squares of
    fixed size per small step, about O(sqrt N), against O(N log N) for the full inverse
    DFT).  The kite at 1024^2, 2048^2, 4096^2 (d = 4, n_c = 8, 8 Gaussians, zero
    Dirichlet data), one large step of 64 small steps per mode after a warm-up call,
    kernels timed with events: per small step the interface evaluation (full: k_ff_cols +
    inverse rows; squares: k_sq_eval) and the U_B step, per large step the whole call."""
    out = {}
    for N in (1024, 2048, 4096):
        name = f"kite{N}"
        w = W.workload(name, d=4, M=7)
        g, p = w.grid, w.params
        plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                              dict(d=4, M=7, B=p.B, k1=p.k1))
        fs = [W.gaussian_sum(w.boundary, 1, 50 + k, wmin=0.05, wmax=0.05, margin=0.35)
              for k in range(n_f)]
        U0 = torch.tensor(np.stack([W.grid_values(w, f) for f in fs]), device=dev)
        u, ut = torch.empty_like(U0), torch.empty_like(U0)
        row = {"grid": f"{N}x{N}", "points": N * N}
        for mode in (False, True):
            u.copy_(U0)
            ut.zero_()
            plan.fc2d_forward_wave(n_f, 1.0, n_c, 1, u, ut, squares=mode)  # builds the band
            u.copy_(U0)
            ut.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.fc2d_forward_wave(n_f, 1.0, n_c, 1, u, ut, squares=mode)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            u.copy_(U0)
            ut.zero_()
            plan.fc2d_profile(True)
            plan.fc2d_profile_read()
            plan.fc2d_forward_wave(n_f, 1.0, n_c, 1, u, ut, squares=mode)
            torch.cuda.synchronize()
            plan.fc2d_profile(False)
            prof = plan.fc2d_profile_read()
            S = 8 * n_c
            per = lambda k: prof[k][1] / prof[k][0] if k in prof else 0.0
            if mode:
                iface = per("sq_eval")
            else:
                iface = per("ff_cols") + per("inverse_rows")
            counts = plan.fc2d_wave_band_info(n_c, squares=mode)
            row["squares" if mode else "full_inverse_dft"] = {
                "ms_per_large_step": ms, "interface_ms_per_small_step": iface,
                "ub_step_ms": per("ub_step"), "unknowns": counts[0], "interface_points": counts[2],
                "n_squares": counts[4]}
        plan.fc2d_destroy()
        out[name] = row
    return {"workload": f"kite N^2, d = 4, n_c = 8, {n_f} Gaussians, one large step (64 small "
                        "steps) per mode, FP64", "n_f": n_f, "by_grid": out}


def stars8_batched(fc2d, torch, dev, replays=10):
    """Eight stars (grids 256^2..2048^2 by concavity), 32 trigonometric sums per domain,
    one fc2d_group_extend_coeffs call per step (one CUDA graph, a branch per domain);
    mixed and FP64.  Inputs are made on the host and copied once; the error is checked
    against the oracle on function 0 of the smallest and of the largest domain."""
    from oracle import fc2d as OF
    from oracle import geometry as OG
    from oracle.fc_matrices import load_fc_matrices
    stars = W.stars8()
    n_f = 32
    inputs = []
    for i, w in enumerate(stars):
        g, p = w.grid, w.params
        probe = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                               dict(B=p.B, k1=p.k1))
        xy = probe.fc2d_boundary_points()
        probe.fc2d_destroy()
        fs = W.star_functions(w, i, n_f)
        xs, ys = g.coords()
        fg = torch.empty((n_f, g.ny, g.nx), dtype=torch.float64, device=dev)
        for m, t in enumerate(fs):
            fg[m].copy_(torch.from_numpy(W.trig_grid(t, xs, ys)))
        fb = torch.tensor(np.stack([t(xy[:, 0], xy[:, 1]) for t in fs]), device=dev)
        inputs.append((w, fs, fg, fb))
    points = n_f * sum(w.grid.nx * w.grid.ny for w in stars)
    out = {"workload": "8 stars r = 1 + a cos k theta, a ~ U[0.1,0.3], k ~ U{3..7} (seed 4), "
                       "grids " + ", ".join(f"{w.grid.nx}^2" for w in sorted(
                           stars, key=lambda s: s.grid.nx)) +
                       ", 32 degree-12 trigonometric sums per domain",
           "points_per_step": points, "unit": UNIT,
           "launch": "fc2d_group_extend_coeffs: one CUDA graph (mixed: the form the "
                     "group's autotuner keeps, see group_tuning; FP64: a branch per domain)"}
    small = min(range(8), key=lambda i: stars[i].grid.nx)
    large = max(range(8), key=lambda i: stars[i].grid.nx)
    for name, prec, dt in (("mixed", fc2d.FC2D_MIXED, torch.float32),
                           ("fp64", fc2d.FC2D_FP64, torch.float64)):
        runs = []
        for w, fs, fg, fb in inputs:
            g, p = w.grid, w.params
            plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                                  dict(B=p.B, k1=p.k1), precision=prec)
            fh = torch.empty((n_f, g.ny, g.nx // 2 + 1, 2), dtype=dt, device=dev)
            runs.append((plan, fg, fb, fh))
        grp = fc2d.fc2d_group_create([r[0] for r in runs])
        gargs = ([n_f] * len(runs), [r[1] for r in runs], [r[2] for r in runs],
                 [r[3] for r in runs])
        for _ in range(3):  # the first call captures the graph, the others replay it
            grp.fc2d_group_extend_coeffs(*gargs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(replays):
            grp.fc2d_group_extend_coeffs(*gargs)
        e1.record()
        torch.cuda.synchronize()
        form, threads, tune_us = grp.fc2d_group_tuning()
        grp.fc2d_group_destroy()
        for plan, *_ in runs:
            plan.fc2d_sync_status()
        ms = e0.elapsed_time(e1) / replays
        errs = {}
        for i in (small, large):
            w, fs, _, _ = inputs[i]
            geo = OG.build_geometry(w)
            st = OF.matching_stencils(geo)
            xs, ys = w.grid.coords()
            ref = OF.coefficients(OF.extension(geo, load_fc_matrices(), W.trig_grid(fs[0], xs, ys),
                                               OF.boundary_values(geo, fs[0]), st))
            got = runs[i][3][0].cpu().numpy().astype(np.float64)
            got = got[..., 0] + 1j * got[..., 1]
            errs[w.name] = float(np.abs(got - ref).max() / np.abs(ref).max())
        out[name] = {"value": points / (ms / 1e3), "ms_per_step": ms, "replays": replays,
                     "err_vs_oracle": errs}
        if threads:
            out[name]["group_tuning"] = {
                "form": form, "queue_threads": threads,
                "us": {k: round(v, 1) for k, v in tune_us.items()},
                "how": "capture-time autotuner: the persistent blend kernel timed with 256 "
                       "and 512 threads per CTA, then the graph with it and the graph with "
                       "a branch per domain timed on the call's inputs; the faster kept"}
        for plan, *_ in runs:
            plan.fc2d_destroy()
    return out


def run_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2010_03901_gb300.build import build
    build()
    from paper_2010_03901_gb300 import fc2d

    w = W.workload(WORKLOAD)
    g, p = w.grid, w.params
    f = bench_functions(w, 1)[0]
    probe = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                           dict(B=p.B, k1=p.k1))
    xy = probe.fc2d_boundary_points()
    probe.fc2d_destroy()
    fg_h = torch.from_numpy(W.grid_values(w, f)).pin_memory()
    fb_h = torch.from_numpy(np.ascontiguousarray(f(xy[:, 0], xy[:, 1]))).pin_memory()

    head = "fp64" if args.precision == "fp64" else "mixed"
    res = {head: measure(fc2d, torch, w, head, args.steps, args.warmup, world, dev, fg_h, fb_h,
                         True)}
    if args.precision == "both":
        k64 = max(3, args.steps // 8)
        res["fp64"] = measure(fc2d, torch, w, "fp64", k64, args.warmup, world, dev, fg_h, fb_h,
                              False)
    r = res[head]
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head == "fp64" else "f32+tf32 (f64 matching values, weights)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": f"{g.nx}x{g.ny}", "normals": p.B,
                       "domain": "kite a=0.65 b=1.5", "functions_per_step": 1,
                       "function": "sum of 16 Gaussians (seed 3)", "precision": head,
                       "d": p.d, "C": p.C, "M": p.M, "n_r": p.n_r,
                       "l2": f"inputs larger than L2: {ROT} rotating copies of f on the "
                             "whole grid (FP64, 134 MB each) and of the spectrum; steps back "
                             "to back (the flushed variant is l2_flushed)",
                       "parallelism": f"replicas x{world}"},
            "clocks": r["clocks"], "roofline": r["roofline"], "kernels": r["kernels"],
            "gpu_launches": r["gpu_launches"], "e2e": r["e2e"], "l2_flushed": r["l2_flushed"],
            "plan_s": r["plan_s"], "tuning": r["tuning"],
            "profiled_ms_per_step": r["profiled_ms_per_step"],
            "kernels_note": "per-kernel times and roofline from a second region of the same "
                            "K steps with CUDA events around each kernel",
            "wall_s_timed": r["wall_s_timed"]}
    if "fp64" in res and head != "fp64":
        q = res["fp64"]
        line["fp64"] = {k: q[k] for k in ("value", "ms_per_step", "profiled_ms_per_step",
                                          "steps", "roofline", "kernels", "e2e", "l2_flushed")}
    if rank == 0 and world == 1 and not args.no_cpu:
        base, spec_ref = cpu_baseline(w)
        line["cpu_baseline"] = base
        for name, q in res.items():
            got = q["fhat"].cpu().numpy().astype(np.float64)
            got = got[..., 0] + 1j * got[..., 1]
            err = float(np.abs(got - spec_ref).max() / np.abs(spec_ref).max())
            if name == head:
                line["err_vs_oracle"] = err
            else:
                line[name]["err_vs_oracle"] = err
    if rank == 0 and world == 1 and not args.no_extra:
        for name in args.extra.split(","):
            line[name] = EXTRA_LINES[name](fc2d, torch, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


EXTRA_LINES = {"poisson_star1024": poisson_star1024,
               "poisson_kite_d10": poisson_kite_oscillatory,
               "ff_interior_kite2048": ff_interior_kite2048,
               "ff_solve_kite2048": ff_solve_kite2048,
               "ff_scaling": ff_scaling,
               "stars8_batched": stars8_batched}


def ff_probe(name):
    """One large step of the Fourier Forwarding solve on workload `name` (d = 4, n_c = 8,
    8 Gaussians, zero Dirichlet data), with the full inverse DFT, the small squares and
    the small squares in double-float: a small, self-contained command for profilers."""
    import torch
    from paper_2010_03901_gb300.build import build
    build()
    from paper_2010_03901_gb300 import fc2d
    w = W.workload(name, d=4, M=7)
    g, p = w.grid, w.params
    plan = fc2d.fc2d_plan(w.boundary.arrays(), (g.a0, g.b0, g.h, g.nx, g.ny),
                          dict(d=4, M=7, B=p.B, k1=p.k1))
    fs = [W.gaussian_sum(w.boundary, 1, 50 + k, wmin=0.05, wmax=0.05, margin=0.35)
          for k in range(8)]
    U0 = torch.tensor(np.stack([W.grid_values(w, f) for f in fs]), device="cuda:0")
    out = {}
    for mode in ("full", "squares", "squares_double_float"):
        u, ut = U0.clone(), torch.zeros_like(U0)
        plan.fc2d_forward_wave(8, 1.0, 8, 1, u, ut, squares=mode != "full",
                               double_float=mode == "squares_double_float")
        plan.fc2d_sync_status()
        out[mode] = float(u.abs().max())
    print(json.dumps({"ff_probe": name, "max_abs_u": out}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--ff-probe", default=None,
                    help="run one Fourier Forwarding large step on this workload and exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fc2d", choices=["fc2d", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: mixed is the headline, FP64 reported beside it")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the Poisson, Fourier Forwarding and batched-star lines")
    ap.add_argument("--extra", default=",".join(EXTRA_LINES),
                    help="comma-separated extra lines to run (default: all of "
                         + ", ".join(EXTRA_LINES) + ")")
    args = ap.parse_args(argv)
    if args.ff_probe:
        ff_probe(args.ff_probe)
        return
    bad = [n for n in args.extra.split(",") if n not in EXTRA_LINES]
    if bad:
        ap.error(f"unknown extra line(s): {', '.join(bad)}")
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
