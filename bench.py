#!/usr/bin/env python
"""Benchmark of the CSR-k SpMV hot path on GB300.

Workload (one "step"): y = A x on two 128^3 stencil matrices, 7-point (n = 2,097,152,
nnz = 14,581,760) and 27-point (nnz = 55,742,968); FP64 values diagonally dominant with
off-diagonals U[-1,0), int32 indices; the input rows/columns carry a random symmetric
permutation (seed 3) that the CSR-k reorder (RCM) undoes; CSR-3 sizes and launch shape
from the library's autotuner; x ~ U[-1,1] (seed 2).  Each step runs, per matrix: permute
x into the reordered numbering, then the CSR-3 kernel storing y in the input numbering
(fused unpermute) -- the whole device path of a natural-numbering csrk_spmv call.  Inputs
are resident in HBM and each step's working set (~930 MB) exceeds the 129 MB L2, so no
flush is needed.  Before timing, every entry of y is checked against the FP64 oracle.

Metric: GFLOP/s (2 flops per stored nonzero per SpMV), whole job over all ranks.
Roofline: HBM bytes of the dominant kernel (the 27-point CSR-3 launch) per launch over its
mean CUDA-event duration, against the measured copy bandwidth (and, beside it, the
nominal 8 TB/s).

Also in the line (outside the timed region): the same step as 100 repeated SpMVs per
matrix replayed from one CUDA graph; the 27-point matrix with values stored FP32 / BF16
(FP32 or FP64 x and accumulation) with each variant's per-entry error against the FP64
oracle; the FEM-like 160^3 matrix; CSR-2 against CSR-3 sizes on the GPU; FP64 against
mixed-precision CG; the 64-matrix batch; and the CPU baseline: the oracle's Listing 1
loop nest with its OpenMP parallel loop on all host cores.

--impl reference times that CPU oracle (Listing 1, OpenMP, all cores) on the same
matrices, RCM-reordered by the oracle, one SpMV of both matrices per step.

Multi-GPU: replicas (one independent copy of the workload per rank, no collective on
the data path); value = all ranks' flops / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

SIDE = 128
# nominal dense FP64 rate of a GB300 (152 SMs x 2 FMA/clock x 2.07 GHz x 2 flops)
FP64_NOMINAL_GFLOPS = 1250.0
# FP64 FMA rate measured on GB300 by a chain-of-independent-FMAs probe: 0.50-0.59 T FMA/s
FP64_PROBE_GFLOPS = (1000.0, 1180.0)
# nominal HBM3e bandwidth of a GB300
NOMINAL_HBM_GBS = 8000.0
WORKLOAD = ("128^3 7-point and 27-point random diagonally dominant stencils (FP64 values, int32 "
            "indices), rows/columns under a random symmetric permutation; y = A x per matrix per step, "
            "x and y in the input numbering")
SR, SSR = 32, 8
MATRICES = (("stencil7", 7), ("stencil27", 27))

# DRAM traffic per launch of the dominant kernel from an ncu capture of the 128^3 launch,
# keyed by (matrix, dtype, kernel number) and valid only for the kernel source it was
# taken on (the profiles directory holds each capture's command and figures).
NCU_TRAFFIC = {
    ("stencil27", "f64", 4): {"bytes": 599_657_728, "kernel_hash": "150e04d362cd"},
    ("stencil27", "f64", 5): {"bytes": 604_811_264, "kernel_hash": "b55ab8bdd2a3"},
}


def kernel_source_hash() -> str:
    """Hash of the FP64 SpMV kernel sources with comments and blank space removed, so that
    a comment edit does not orphan a capture of unchanged code."""
    import re
    h = hashlib.sha1()
    for f in ("kernels.cuh", "launch_impl.cuh", "spmv_f64.cu"):
        with open(os.path.join(ROOT, "paper_2203_05096_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:12]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, dist=None, device="cpu"):
    """Slowest rank's time (the job is done when the last replica is); `dist` may be None."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Units all replicas processed per second, over the slowest replica's time."""
    return world * units_per_rank / (ms * 1e-3)


def build_matrices(side=SIDE, only=None):
    n = side ** 3
    labels = synth.vectors.permutation(n, 3)
    out = []
    for name, pts in MATRICES:
        if only and name != only:
            continue
        out.append((name, synth.stencil_3d(side, side, side, pts, "random_dd", 3, labels=labels)))
    return out


def alg_bytes_spmv(n, nnz, nsr, nssr, val_bytes=8, x_bytes=8, fused_unpermute=True, col_bytes=4, runs=0,
                   row_order=False):
    # every stored value and column index (4 bytes, or a 2-byte code with kernels 4 to 6),
    # rowptr, sr_ptr, the 32-byte SSR descriptors, x read once and y written once
    # (beta = 0), the permutation read once when the kernel stores y in the input
    # numbering, and for kernels 5 / 6 the run table (8 bytes per run of x, a 4-byte run
    # pointer per SSR) and the rows' length order when it is used (2 bytes per row)
    return ((val_bytes + col_bytes) * nnz + 4 * (n + 1) + 4 * (nsr + 1) + 32 * nssr + x_bytes * n + x_bytes * n
            + (4 * n if fused_unpermute else 0) + (8 * runs + 4 * (nssr + 1) if runs else 0)
            + (2 * n if row_order else 0))


def col_bytes_of(cfg):
    return 2 if cfg.get("kernel") in (4, 5, 6) else 4


def window_of(h, cfg):
    """Kernels 5 / 6: (run count, whether the row length order is used); (0, False) otherwise."""
    if cfg.get("kernel") not in (5, 6):
        return 0, False
    from paper_2203_05096_gb300 import csrk
    w = csrk.xwin_info(h)
    return w["runs"], w["row_order"]


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            p = [t.strip() for t in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def visible_gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def cpu_reordered(mats):
    """Each matrix under the oracle's own RCM ordering (B = P A P^T), the form the CPU
    CSR-k loop nest runs on, as the GPU path does."""
    from oracle import reorder
    out = []
    for name, a in mats:
        p = reorder.rcm(a.n, a.rowptr, a.colidx)
        rp, ci, v = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, p)
        out.append((name, a.n, rp, ci, v))
    return out


def cpu_listing1(rmats, sr, ssr, warm=5, runs=20, threads=0):
    """The oracle's Listing 1 loop nest with its OpenMP parallel loop over super-super-rows
    (static schedule) on the host cores: 5 untimed warm-ups and the mean of 20 timed runs
    per matrix (the paper's CPU methodology, Sec. 5.4).  Returns (GFLOP/s over both
    matrices, threads used, seconds timed)."""
    from oracle import csrk as ocsrk
    from oracle import spmv as ospmv
    flops, secs, used = 0.0, 0.0, 1
    for name, n, rp, ci, v in rmats:
        sr_ptr, ssr_ptr = ocsrk.fixed_pointers(n, sr, ssr)
        x = synth.uniform_vector(n, 2)
        y = np.empty(n)
        for _ in range(warm):
            _, used = ospmv.csr3_spmv_omp(ssr_ptr, sr_ptr, rp, ci, v, x, threads, out=y)
        t0 = time.perf_counter()
        for _ in range(runs):
            ospmv.csr3_spmv_omp(ssr_ptr, sr_ptr, rp, ci, v, x, threads, out=y)
        secs += time.perf_counter() - t0
        flops += runs * 2.0 * float(rp[-1])
    return flops / secs / 1e9, used, secs


def cpu_section(mats):
    """CPU baseline and the host half of the CSR-2 / CSR-3 comparison (Sec. 6.1): the
    paper's constant-time CPU choice CSR-2 with 96-row super-rows (Sec. 4.2) is the
    baseline; a few other CSR-2 super-row sizes and CSR-3 shapes beside it, and the plain
    single-thread CSR oracle for reference."""
    from oracle import spmv as ospmv
    t0 = time.perf_counter()
    rm = cpu_reordered(mats)
    prep = time.perf_counter() - t0
    g96, used, secs = cpu_listing1(rm, 96, 1)
    study = {"csr2": {}, "csr3": {}}
    for srs in (32, 384, 1536):
        study["csr2"][str(srs)] = round(cpu_listing1(rm, srs, 1)[0], 2)
    study["csr2"]["96"] = round(g96, 2)
    for sr, ssr in ((32, 4), (96, 4), (32, 32)):
        study["csr3"][f"{sr}x{ssr}"] = round(cpu_listing1(rm, sr, ssr)[0], 2)
    # the plain single-thread oracle loop, whole matrices, two passes each
    fl, t1 = 0.0, time.perf_counter()
    for name, n, rp, ci, v in rm:
        x = synth.uniform_vector(n, 2)
        for _ in range(2):
            ospmv.csr_spmv(n, rp, ci, v, x)
            fl += 2.0 * float(rp[-1])
    study["plain_csr_1_thread"] = round(fl / (time.perf_counter() - t1) / 1e9, 3)
    study["threads"] = used
    study["host_cores"] = os.cpu_count()
    base = {"value": round(g96, 3), "unit": "GFLOP/s", "cores": used, "kind": "oracle",
            "sample": f"Listing 1 loop nest (oracle C, OpenMP static over super-super-rows), CSR-2 with "
                      f"96-row super-rows, both 128^3 matrices RCM-reordered by the oracle ({prep:.0f} s), "
                      f"5 warm-ups + 20 timed SpMVs each ({secs:.2f} s timed)"}
    return base, study


# ------------------------------------------------------------------ our arm
def max_norm_err(got, ref, s):
    """max_i |got_i - ref_i| / s_i (rows with s_i = 0 must match exactly: inf otherwise)."""
    err = np.abs(got - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(s > 0, err / np.where(s > 0, s, 1.0), np.where(err > 0, np.inf, 0.0))
    return float(np.max(q)) if q.size else 0.0


def check_every_row(a, x, got, bound, what):
    """Every entry of y against the FP64 oracle (Sec. 1's y = A x, Listing 1's row loop)."""
    from oracle import spmv as ospmv
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    s = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x)
    e = max_norm_err(got, ref, s)
    if not e <= bound:
        raise RuntimeError(f"{what}: result check failed before timing (max normalised error {e:.3e})")
    return e


def event_pair():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_graph_100(state, stream, perm_fn, spmv_fn, XP, reps=3):
    """The benchmark step as 100 repeated SpMVs per matrix (permute x + CSR-3 kernel),
    recorded once into a CUDA graph and replayed; mean time per SpMV."""
    import torch
    out = {}
    for s in state:
        h = s["h"]
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            # warm the capture stream (first launches on a stream may set attributes)
            perm_fn(h, 0, 1, s["x"].data_ptr(), 1, s["xp"].data_ptr(), 1, 0, cap.cuda_stream)
            spmv_fn(h, 1.0, s["xp"].data_ptr(), 0.0, s["y"].data_ptr(), XP, cap.cuda_stream)
            cap.synchronize()
            with torch.cuda.graph(g, stream=cap):
                rc = 0
                for _ in range(100):
                    rc |= perm_fn(h, 0, 1, s["x"].data_ptr(), 1, s["xp"].data_ptr(), 1, 0, cap.cuda_stream)
                    rc |= spmv_fn(h, 1.0, s["xp"].data_ptr(), 0.0, s["y"].data_ptr(), XP, cap.cuda_stream)
        torch.cuda.current_stream().wait_stream(cap)
        if rc:
            raise RuntimeError("graph capture of the SpMV loop failed")
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = event_pair()
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / (reps * 100) * 1e3
        out[s["name"]] = {"us_per_spmv": round(us, 2), "gflops": round(2.0 * s["a"].nnz / (us * 1e-6) / 1e9, 1)}
        del g
    return out


def time_kernel(h, xp, y, flags, stream, reps=50, x_f32=False):
    """Mean CUDA-event time of the CSR-3 kernel alone (x already in the reordered numbering,
    y stored through the permutation), in microseconds."""
    from paper_2203_05096_gb300 import csrk
    f = flags | (csrk.X_F32 if x_f32 else 0)
    for _ in range(3):
        csrk.spmv(h, 1.0, xp, 0.0, y, f)
    import torch
    torch.cuda.synchronize()
    e0, e1 = event_pair()
    e0.record(stream)
    for _ in range(reps):
        csrk.spmv(h, 1.0, xp, 0.0, y, f)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e3


def run_precision(a, s64, dev, stream, peak):
    """The 27-point matrix with values stored FP64 / FP32 / BF16 and x, accumulation in FP64
    or FP32: kernel time, bytes and roofline fraction, and each variant's per-entry error
    against the FP64 oracle (FP64 values, FP64 x), normalised by s_i = sum_j |a_ij x_j|."""
    import torch
    from oracle import spmv as ospmv
    from paper_2203_05096_gb300 import csrk
    x = synth.uniform_vector(a.n, 2)
    ref = ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x)
    sc = ospmv.abs_row_scale(a.rowptr, a.colidx, a.vals, x)
    out = {"matrix": "stencil27", "error": "max_i |y_i - y64_i| / sum_j |a_ij x_j| against the FP64 oracle"}
    variants = (("f64", False, False), ("f32", False, False), ("f32", True, False), ("f32", True, True),
                ("bf16", False, False), ("bf16", True, True))
    handles = {"f64": s64["h"]}
    for dt, x32, acc32 in variants:
        if dt not in handles:
            h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dt)
            csrk.reorder(h, "rcm", want_perm=False)
            csrk.set_sizes(h, 0, 0)
            handles[dt] = h
        h = handles[dt]
        xt = torch.tensor(x, dtype=torch.float32 if x32 else torch.float64, device=dev)
        xp, y = torch.empty_like(xt), torch.empty_like(xt)
        csrk.permute(h, 0, 1, xt, 1, xp, 1, csrk.X_F32 if x32 else 0)
        fl = csrk.X_PERMUTED | (csrk.ACC_F32 if acc32 else 0)
        us = time_kernel(h, xp, y, fl, stream, x_f32=x32)
        got = y.double().cpu().numpy()
        inf, cfg = csrk.info(h), csrk.tuned_config(h)
        vb = {"f64": 8, "f32": 4, "bf16": 2}[dt]
        runs, ro = window_of(h, cfg)
        ab = alg_bytes_spmv(inf["n"], inf["nnz"], inf["nsr"], inf["nssr"], vb, 4 if x32 else 8,
                            col_bytes=col_bytes_of(cfg), runs=runs, row_order=ro)
        key = f"{dt}_x{'32' if x32 else '64'}_acc{'32' if acc32 else '64'}"
        out[key] = {"kernel_us": round(us, 2), "gflops": round(2.0 * a.nnz / (us * 1e-6) / 1e9, 1),
                    "gbs": round(ab / (us * 1e-6) / 1e9, 1), "frac_of_peak": round(ab / (us * 1e-6) / 1e9 / peak, 3),
                    "max_err": float(f"{max_norm_err(got, ref, sc):.3e}"), "kernel": cfg["kernel"]}
    for dt, h in handles.items():
        if dt != "f64":
            csrk.destroy(h)
    return out


def run_k_study(entries, stream):
    """CSR-2 (one super-row per super-super-row) against CSR-3 sizes on the GPU, each size
    pair with the matrix's tuned kernel and launch shape (Sec. 6.2 / 7): kernel time."""
    from paper_2203_05096_gb300 import csrk
    out = {}
    for name, h, xp, y in entries:
        cfg = csrk.tuned_config(h)
        row = {}
        for sr, ssr in ((32, 1), (64, 1), (128, 1), (32, 2), (32, 4), (32, 8)):
            csrk.set_sizes(h, sr, ssr)
            csrk.set_config(h, kernel=cfg["kernel"], lanes=cfg["lanes"], unroll=cfg["unroll"], warps=cfg["warps"],
                            stages=0, ctas=0)
            try:
                row[f"{sr}x{ssr}"] = round(time_kernel(h, xp, y, csrk.X_PERMUTED, stream, reps=30), 1)
            except csrk.CsrkError:
                row[f"{sr}x{ssr}"] = None   # does not fit the forced kernel's stages
        out[name] = row
    return out


def run_ours(args, world, rank, local):
    import ctypes  # noqa: F401

    import torch
    from paper_2203_05096_gb300 import csrk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lib = csrk.lib()
    mats = build_matrices(args.side, args.only)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    state = []
    for name, a in mats:
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, args.dtype)
        t_order = time.perf_counter()
        if args.ordering == "bandk":      # Band-k with its own variable SR / SSR pointers
            csrk.reorder_bandk(h, *(int(v) for v in args.bandk_caps.split(",")), want_perm=False)
        else:
            csrk.reorder(h, "rcm", want_perm=False)
        t_order = time.perf_counter() - t_order
        t_tune = time.perf_counter()
        if args.sizes == "auto":
            csrk.set_sizes(h, 0, 0)          # the library's autotuner (timed on this matrix)
        else:
            csrk.set_sizes(h, *(int(v) for v in args.sizes.split(",")))
        t_tune = time.perf_counter() - t_tune
        if args.config:
            csrk.set_config(h, **{k: int(v) for k, v in (kv.split("=") for kv in args.config.split(","))})
        inf = csrk.info(h)
        x = torch.tensor(synth.uniform_vector(a.n, 2), dtype=torch.float64, device=dev)
        xp, yp, y = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        cfg = csrk.tuned_config(h)
        runs, ro = window_of(h, cfg)
        state.append(dict(name=name, a=a, h=h, info=inf, x=x, xp=xp, yp=yp, y=y, cfg=cfg,
                          runs=runs, row_order=ro, tune_s=t_tune, order_s=t_order))

    perm_fn, spmv_fn = lib.csrk_permute, lib.csrk_spmv
    XP = csrk.X_PERMUTED   # x in the reordered numbering, y stored to its input place

    def step(events=None, i=0):
        for j, s in enumerate(state):
            h = s["h"]
            if events is not None:
                events[j][2][i].record(stream)
            rc = perm_fn(h, 0, 1, s["x"].data_ptr(), 1, s["xp"].data_ptr(), 1, 0, sp)
            if events is not None:
                events[j][0][i].record(stream)
            rc |= spmv_fn(h, 1.0, s["xp"].data_ptr(), 0.0, s["y"].data_ptr(), XP, sp)
            if events is not None:
                events[j][1][i].record(stream)
            if rc:
                raise RuntimeError(lib.csrk_last_error().decode())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness guard before timing: every entry of y of the timed launch configuration
    guard = {}
    for s in state:
        tol = 1e-12 if args.dtype == "f64" else 2.0 ** -8
        guard[s["name"]] = check_every_row(s["a"], s["x"].cpu().numpy(), s["y"].cpu().numpy(), tol, s["name"])

    K = args.steps
    events = [[[torch.cuda.Event(enable_timing=True) for _ in range(K)] for _ in range(3)] for _ in state]
    t_start, t_end = event_pair()
    sampler = ClockSampler(visible_gpu_index(local))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    torch.cuda.synchronize()
    t_start.record(stream)
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler keep only the timed launches
    for i in range(K):
        step(events, i)
    torch.cuda.nvtx.range_pop()
    t_end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    kern_ms = [[events[j][0][i].elapsed_time(events[j][1][i]) for i in range(K)] for j in range(len(state))]
    perm_ms = [[events[j][2][i].elapsed_time(events[j][0][i]) for i in range(K)] for j in range(len(state))]
    ms = max_over_ranks(ms, dist, dev)
    status = sum(csrk.device_status(s["h"]) for s in state)
    if status:
        raise RuntimeError("device status word set during the timed region")

    flops_step = sum(2.0 * s["a"].nnz for s in state)
    value = whole_job_rate(world, K * flops_step, ms) / 1e9

    # roofline of the dominant kernel: the 27-point CSR-3 launch
    peak, peak_kind = measured_peaks()
    vb = {"f64": 8, "f32": 4, "bf16": 2}[args.dtype]

    def bytes_of(s):
        inf = s["info"]
        return alg_bytes_spmv(inf["n"], inf["nnz"], inf["nsr"], inf["nssr"], vb, col_bytes=col_bytes_of(s["cfg"]),
                              runs=s["runs"], row_order=s["row_order"])

    dom = max(range(len(state)), key=lambda j: statistics.mean(kern_ms[j]))
    sd = state[dom]
    abytes = bytes_of(sd)
    kmean = statistics.mean(kern_ms[dom])
    achieved = abytes / (kmean * 1e-3) / 1e9
    khash = kernel_source_hash()
    tr = NCU_TRAFFIC.get((sd["name"], args.dtype, sd["cfg"]["kernel"]))
    traffic = tr["bytes"] if tr and tr["kernel_hash"] == khash else None

    per_matrix = {}
    for j, s in enumerate(state):
        km = statistics.mean(kern_ms[j])
        b = bytes_of(s)
        gbs = b / (km * 1e-3) / 1e9
        c = s["cfg"]
        per_matrix[s["name"]] = {"kernel_us": round(km * 1e3, 2), "kernel_min_us": round(min(kern_ms[j]) * 1e3, 2),
                                 "gbs": round(gbs, 1), "frac_of_peak": round(gbs / peak, 3),
                                 "frac_of_nominal": round(gbs / NOMINAL_HBM_GBS, 3),
                                 "gflops": round(2.0 * s["info"]["nnz"] / (km * 1e-3) / 1e9, 1),
                                 "permute_us": round(statistics.mean(perm_ms[j]) * 1e3, 2),
                                 "alg_bytes": int(b), "sizes": [s["info"]["sr"], s["info"]["ssr"]],
                                 "x_runs": int(s["runs"]),
                                 "shape": f"k{c['kernel']} u{c['unroll']} w{c['warps']} s{c['stages']} c{c['ctas']}",
                                 "max_err": float(f"{guard[s['name']]:.2e}")}

    # end to end: the public call with host vectors (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hx = [torch.tensor(synth.uniform_vector(s["a"].n, 2), dtype=torch.float64).pin_memory() for s in state]
        hy = [torch.empty(s["a"].n, dtype=torch.float64).pin_memory() for s in state]
        HV = csrk.HOST_VECTORS
        E = max(5, min(args.steps // 10, 200))

        def e2e_step():
            for j, s in enumerate(state):
                if spmv_fn(s["h"], 1.0, hx[j].data_ptr(), 0.0, hy[j].data_ptr(), HV, sp):
                    raise RuntimeError(lib.csrk_last_error().decode())
        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = event_pair()
        e0.record(stream)
        for _ in range(E):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        e2e = {"value": round(whole_job_rate(world, E * flops_step, ems) / 1e9, 2), "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(sum(8 * s["a"].n for s in state)),
               "d2h_bytes_per_step": int(sum(8 * s["a"].n for s in state))}

    graph = None
    if not args.no_graph:
        graph = run_graph_100(state, stream, perm_fn, spmv_fn, XP)

    # conjugate gradients to rtol 1e-10 on the 27-point matrix: FP64 against mixed precision
    cg = None
    s27 = next((s for s in state if s["name"] == "stencil27"), None)
    if not args.no_cg and s27 is not None:
        b = torch.tensor(synth.uniform_vector(s27["a"].n, 5), dtype=torch.float64, device=dev)
        xs = torch.empty_like(b)
        cg = {"matrix": s27["name"], "rtol": 1e-10, "replace_every": 20, "runs": {}}
        for inner, restart in (("f64", 0), ("f32", 0), ("bf16", 1)):
            csrk.cg(s27["h"], b, xs, 1e-10, 5000, inner, 20, restart)     # capture the graphs
            torch.cuda.synchronize()
            times = []
            for rep in range(3):
                c0, c1 = event_pair()
                c0.record(stream)
                if rep == 0:
                    torch.cuda.nvtx.range_push(f"cg_{inner}")   # lets a profiler keep one solve
                rc, iters, rel = csrk.cg(s27["h"], b, xs, 1e-10, 5000, inner, 20, restart)
                if rep == 0:
                    torch.cuda.nvtx.range_pop()
                c1.record(stream)
                torch.cuda.synchronize()
                times.append(c0.elapsed_time(c1))
            cg["runs"][inner] = {"ms": round(min(times), 3), "ms_median": round(statistics.median(times), 3),
                                 "iterations": iters, "true_relres": rel, "converged": rc == 0,
                                 "restart": restart}
        f64 = cg["runs"]["f64"]["ms"]
        for k in ("f32", "bf16"):
            cg["runs"][k]["speedup_vs_f64"] = round(f64 / cg["runs"][k]["ms"], 3)

    precision = None
    if not args.no_precision and s27 is not None and args.dtype == "f64":
        precision = run_precision(s27["a"], s27, dev, stream, peak)

    fem, fem_entry = None, None
    if not args.no_fem and args.side == SIDE:
        fem, fem_entry = run_fem(args, dev, keep=True)

    k_study = None
    if not args.no_kstudy:
        entries = [(s["name"], s["h"], s["xp"], s["y"]) for s in state]
        if fem_entry is not None:
            entries.append(fem_entry)
        k_study = run_k_study(entries, stream)
    if fem_entry is not None:
        csrk.destroy(fem_entry[1])

    batch = None
    if not args.no_batch:
        batch = run_batch(args, dev, stream, peak)

    cpu, cpu_study = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, cpu_study = cpu_section(mats)

    if rank == 0:
        line = {
            "metric": "SpMV GFLOP/s (CSR-3, 128^3 7-point + 27-point stencils, FP64)",
            "value": round(value, 2),
            "unit": "GFLOP/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": round(ms / K, 5),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": args.dtype,
            "data": "synthetic",
            "config": {"workload": "128^3 7-pt + 27-pt stencils, FP64, int32, random labels undone by RCM",
                       "l2": "inputs larger than L2 (~930 MB per step vs 129 MB), no flush",
                       "sizes": args.sizes, "ordering": args.ordering if args.ordering == "rcm" else
                       f"bandk {args.bandk_caps}", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": f"csr3 {sd['name']}",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "alg_bytes_per_launch": int(abytes), "peak_kind": peak_kind,
                         "nominal_gbs": NOMINAL_HBM_GBS, "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                         "kernel_hash": khash,
                         # the same launch against GB300's FP64 FMA rate (one FMA per nonzero):
                         # the SpMV is co-bound by HBM and the FP64 pipe
                         "fp64": {"achieved_gflops": round(2.0 * sd["info"]["nnz"] / (kmean * 1e-3) / 1e9, 1),
                                  "nominal_gflops": FP64_NOMINAL_GFLOPS, "probe_gflops": list(FP64_PROBE_GFLOPS),
                                  "frac_of_nominal": round(2.0 * sd["info"]["nnz"] / (kmean * 1e-3) / 1e9
                                                           / FP64_NOMINAL_GFLOPS, 4)}},
            "e2e": e2e,
            "batch": batch,
            "cg": cg,
            "wall_s_timed": round(wall, 3),
            "gpu_launches": K * 2 * len(state),   # per matrix: permute x, CSR-3 kernel (+ fused unpermute)
            "clocks": clocks,
            "per_matrix": per_matrix,
            "graph_100": graph,
            "precision": precision,
            "fem": fem,
            "k_study_gpu_us": k_study,
            "cpu_study_gflops": cpu_study,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    for s in state:
        csrk.destroy(s["h"])
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ batched workload
def run_batch(args, dev, stream, peak):
    """64 stencil / FEM matrices, n log-uniform in [1e3, 1e6] (seed 6), FP64 and FP32 values,
    k in {1,2,4,8,16} right-hand sides; sizes from the autotuner; one persistent SpMM
    launch per step, then 200 CG iterations recorded in one CUDA graph, then CG to a 1e-10
    true residual with the FP64 operator, plain FP64 vs mixed precision."""
    import torch
    from paper_2203_05096_gb300 import csrk
    specs = synth.batch_specs()
    t0 = time.perf_counter()
    hs, mats = [], []
    for sp in specs:
        a = synth.batch_matrix(sp)
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, sp["dtype"])
        csrk.reorder(h, "rcm", want_perm=False)
        csrk.set_sizes(h, 0, 0)
        hs.append(h)
        mats.append((a.n, a.nnz, sp))
    setup_s = time.perf_counter() - t0
    ks = [sp["k"] for sp in specs]
    b = csrk.batch_create(hs, ks)
    Xs = [torch.tensor(synth.uniform_block(n, sp["k"], 500 + i), device=dev) for i, (n, _, sp) in enumerate(mats)]
    Ys = [torch.empty_like(x) for x in Xs]
    for _ in range(3):
        csrk.batch_spmm(b, 1.0, Xs, 0.0, Ys)
    torch.cuda.synchronize()
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        csrk.batch_spmm(b, 1.0, Xs, 0.0, Ys)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = sum(2.0 * nnz * sp["k"] for (n, nnz, sp) in mats)
    vbytes = sum(({"f64": 8, "f32": 4}[sp["dtype"]] + 4) * nnz + 4 * (n + 1) + 16 * n * sp["k"]
                 for (n, nnz, sp) in mats)
    out = {"matrices": len(mats), "n_total": int(sum(m[0] for m in mats)),
           "nnz_total": int(sum(m[1] for m in mats)), "systems": int(sum(ks)), "setup_s": round(setup_s, 1),
           "spmm_ms": round(ms, 4), "spmm_gflops": round(flops / (ms * 1e-3) / 1e9, 1),
           "spmm_gbs": round(vbytes / (ms * 1e-3) / 1e9, 1),
           "spmm_frac_of_peak": round(vbytes / (ms * 1e-3) / 1e9 / peak, 3), "launches_per_step": 1,
           # k > 1 makes the batch FP64-FMA bound: k FMAs per stored nonzero
           "spmm_bound": "fp64", "fp64_peak_gflops": FP64_NOMINAL_GFLOPS,
           "spmm_frac_of_fp64": round(flops / (ms * 1e-3) / 1e9 / FP64_NOMINAL_GFLOPS, 3),
           "plan": csrk.batch_plan(b)}
    # the same product in FP32 arithmetic (values rounded to FP32, FP32 vectors and
    # accumulation): memory-bound, the inner product of the mixed-precision solve
    X32 = [x.float() for x in Xs]
    Y32 = [torch.empty_like(x) for x in X32]
    f32 = csrk.VEC_PERMUTED | csrk.X_F32 | csrk.ACC_F32
    for _ in range(3):
        csrk.batch_spmm(b, 1.0, X32, 0.0, Y32, flags=f32)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        csrk.batch_spmm(b, 1.0, X32, 0.0, Y32, flags=f32)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1) / reps
    vbytes32 = sum(({"f64": 4, "f32": 4, "bf16": 2}[sp["dtype"]] + 4) * nnz + 4 * (n + 1) + 8 * n * sp["k"]
                   for (n, nnz, sp) in mats)
    out["spmm_f32"] = {"ms": round(ms32, 4), "gflops": round(flops / (ms32 * 1e-3) / 1e9, 1),
                       "gbs": round(vbytes32 / (ms32 * 1e-3) / 1e9, 1), "bound": "hbm",
                       "frac_of_peak": round(vbytes32 / (ms32 * 1e-3) / 1e9 / peak, 3)}
    if args.no_cg:
        csrk.batch_destroy(b)
        for h in hs:
            csrk.destroy(h)
        return out
    Bs = [torch.tensor(synth.uniform_block(n, sp["k"], 700 + i), device=dev) for i, (n, _, sp) in enumerate(mats)]
    Xc = [torch.zeros_like(x) for x in Bs]
    csrk.batch_cg(b, Bs, Xc, 200, 1e-10)          # records the 200-iteration graph
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    rel, its = csrk.batch_cg(b, Bs, Xc, 200, 1e-10)
    c1.record(stream)
    torch.cuda.synchronize()
    out["cg"] = {"iterations_in_graph": 200, "ms": round(c0.elapsed_time(c1), 3),
                 "converged_systems": int(np.sum(rel <= 1e-10)), "max_relres": float(np.max(rel)),
                 "median_iterations": float(np.median(its))}
    # time to a 1e-10 true residual on every system, FP64 operator: plain FP64 CG vs mixed
    # precision (FP32 / BF16 inner products, FP64 residual every 20 iterations)
    solve = {}
    for inner in ("f64", "f32", "bf16"):
        Xs = [torch.zeros_like(x) for x in Bs]
        rst = 1 if inner == "bf16" else 0     # BF16: restart p = r at every replacement
        csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=2000, inner=inner, restart=rst)   # records the graph
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        torch.cuda.nvtx.range_push(f"solve_{inner}")   # lets a profiler keep one solve's launches
        rc, rel, its, cycles = csrk.batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=2000, inner=inner, restart=rst)
        torch.cuda.nvtx.range_pop()
        s1.record(stream)
        torch.cuda.synchronize()
        solve[inner] = {"ms": round(s0.elapsed_time(s1), 3), "converged_systems": int(np.sum(rel <= 1e-10)),
                        "all_converged": rc == 0, "max_relres": float(np.max(rel)), "cycles": cycles,
                        "median_iterations": float(np.median(its)), "max_iterations": int(np.max(its))}
    for inner in ("f32", "bf16"):
        solve[inner]["speedup_vs_f64"] = round(solve["f64"]["ms"] / solve[inner]["ms"], 3)
    out["cg_solve"] = {"rtol": 1e-10, "replace_every": 20, "runs": solve}
    csrk.batch_destroy(b)
    for h in hs:
        csrk.destroy(h)
    return out


# ------------------------------------------------------------------ irregular matrices
def run_irregular(args, dev):
    """A 100^3 7-point stencil (random labels) plus 16 coupling rows of 100,000 entries:
    SpMV (natural numbering, fused unpermute) with the long rows left in the super-rows
    versus moved out by csrk_split_long_rows, both autotuned."""
    import torch
    from paper_2203_05096_gb300 import csrk
    side = 100
    n = side ** 3
    base = synth.stencil_3d(side, side, side, 7, "random_dd", 3, labels=synth.vectors.permutation(n, 3))
    a = synth.with_dense_rows(base, 16, 100_000, 7)
    x = torch.tensor(synth.uniform_vector(n, 2), dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "100^3 7-point stencil + 16 coupling rows of 100,000 entries (random labels)",
           "n": n, "nnz": int(a.nnz), "max_row": int(a.row_lengths().max())}
    for mode in ("in_super_rows", "split"):
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
        csrk.reorder(h, "rcm", want_perm=False)
        nl = csrk.split_long_rows(h, 4096) if mode == "split" else 0
        csrk.set_sizes(h, 0, 0)
        for _ in range(5):
            csrk.spmv(h, 1.0, x, 0.0, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(50):
            csrk.spmv(h, 1.0, x, 0.0, y)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / 50 * 1e3
        out[mode] = {"us": round(us, 2), "gflops": round(2.0 * a.nnz / (us * 1e-6) / 1e9, 1), "long_rows": nl,
                     "config": csrk.tuned_config(h)}
        csrk.destroy(h)
    out["speedup"] = round(out["in_super_rows"]["us"] / out["split"]["us"], 2)
    return out


def run_fem(args, dev, keep=False):
    """The FEM-like SPD matrix on 160^3 jittered points (n = 4,096,000, ~61 M nonzeros,
    12-18 neighbours per row, random labels): natural-numbering SpMV (permute x, CSR-3
    kernel with the fused unpermute), autotuned; kernel time with CUDA events, the same
    algorithmic-byte roofline as the stencils, and every entry of y against the FP64
    oracle.  With keep, also returns (name, handle, x_p, y) for the size study."""
    import torch
    from paper_2203_05096_gb300 import csrk
    t0 = time.perf_counter()
    a = synth.fem_like(160, 4)
    gen_s = time.perf_counter() - t0
    xh = synth.uniform_vector(a.n, 2)
    x = torch.tensor(xh, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h, "rcm", want_perm=False)
    csrk.set_sizes(h, 0, 0)
    for _ in range(5):
        csrk.spmv(h, 1.0, x, 0.0, y)
    torch.cuda.synchronize()
    err = check_every_row(a, xh, y.cpu().numpy(), 1e-12, "FEM 160^3")
    reps = max(20, args.steps)
    e0, e1 = event_pair()
    e0.record(stream)
    for _ in range(reps):
        csrk.spmv(h, 1.0, x, 0.0, y)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / reps * 1e3
    inf, cfg = csrk.info(h), csrk.tuned_config(h)
    peak, peak_kind = measured_peaks()
    # kernel alone (x already permuted; y stored through the permutation)
    xp = torch.empty_like(x)
    csrk.permute(h, 0, 1, x, 1, xp, 1)
    kus = time_kernel(h, xp, y, csrk.X_PERMUTED, stream, reps=reps)
    runs, ro = window_of(h, cfg)
    ab = alg_bytes_spmv(inf["n"], inf["nnz"], inf["nsr"], inf["nssr"], 8, col_bytes=col_bytes_of(cfg), runs=runs,
                        row_order=ro)
    out = {"n": int(a.n), "nnz": int(a.nnz), "generate_s": round(gen_s, 1),
           "sizes": [inf["sr"], inf["ssr"]],
           "shape": f"k{cfg['kernel']} u{cfg['unroll']} w{cfg['warps']} s{cfg['stages']} c{cfg['ctas']}",
           "call_us": round(us, 2), "call_gflops": round(2.0 * a.nnz / (us * 1e-6) / 1e9, 1),
           "kernel_us": round(kus, 2), "kernel_gflops": round(2.0 * a.nnz / (kus * 1e-6) / 1e9, 1),
           "kernel_alg_bytes": int(ab), "kernel_gbs": round(ab / (kus * 1e-6) / 1e9, 1),
           "kernel_frac_of_peak": round(ab / (kus * 1e-6) / 1e9 / peak, 3), "max_err": float(f"{err:.2e}")}
    if keep:
        return out, ("fem160", h, xp, y)
    csrk.destroy(h)
    return out


# ------------------------------------------------------------------ reference arm
def run_reference(args, world, rank, local):
    """The FP64 CPU oracle as it stands: Listing 1's loop nest with its OpenMP parallel loop
    over super-super-rows, on all host cores, over both matrices RCM-reordered by the
    oracle; CSR-2 with 96-row super-rows (Sec. 4.2's constant-time CPU choice).  One step =
    one SpMV of each matrix (the whole workload)."""
    if rank != 0:
        return
    from oracle import csrk as ocsrk
    from oracle import spmv as ospmv
    mats = build_matrices(args.side, args.only)
    t0 = time.perf_counter()
    rm = cpu_reordered(mats)
    prep = time.perf_counter() - t0
    work = []
    for name, n, rp, ci, v in rm:
        sr_ptr, ssr_ptr = ocsrk.fixed_pointers(n, 96, 1)
        work.append((sr_ptr, ssr_ptr, rp, ci, v, synth.uniform_vector(n, 2), np.empty(n)))
    used = 1

    def step():
        nonlocal used
        fl = 0.0
        for sr_ptr, ssr_ptr, rp, ci, v, x, y in work:
            _, used = ospmv.csr3_spmv_omp(ssr_ptr, sr_ptr, rp, ci, v, x, 0, out=y)
            fl += 2.0 * float(rp[-1])
        return fl

    for _ in range(args.warmup):
        step()
    flops = 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flops += step()
    dt = time.perf_counter() - t0
    value = flops / dt / 1e9
    sample = (f"every row of both {args.side}^3 matrices per step (RCM by the oracle, {prep:.0f} s before timing), "
              f"Listing 1 loop nest, CSR-2 with 96-row super-rows, OpenMP static, {args.steps} steps in {dt:.2f} s")
    line = {
        "impl": "reference",
        "metric": "SpMV GFLOP/s (CSR-3, 128^3 7-point + 27-point stencils, FP64)",
        "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "128^3 7-pt + 27-pt stencils, FP64, int32, random labels undone by RCM",
                   "method": "FP64 CPU oracle: Listing 1 loop nest with OpenMP over super-super-rows"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--dtype", choices=("f64", "f32", "bf16"), default="f64")
    p.add_argument("--config", default="", help="force a launch config, e.g. kernel=0,lanes=1,warps=8")
    p.add_argument("--sizes", default="auto", help="'auto' (autotuner) or 'sr,ssr'")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cg", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="skip the 100-SpMV CUDA-graph replay")
    p.add_argument("--no-precision", action="store_true", help="skip the FP32/BF16-value variants")
    p.add_argument("--no-fem", action="store_true", help="skip the FEM 160^3 matrix")
    p.add_argument("--no-kstudy", action="store_true", help="skip the CSR-2 / CSR-3 size study")
    p.add_argument("--quick", action="store_true",
                   help="headline step only (no e2e, graph, CG, precision, FEM, size study, batch, CPU)")
    p.add_argument("--side", type=int, default=SIDE, help="grid side (profiling runs use a smaller case)")
    p.add_argument("--only", choices=[m for m, _ in MATRICES], default=None)
    p.add_argument("--ordering", choices=("rcm", "bandk"), default="rcm",
                   help="row ordering: RCM with fixed sizes, or Band-k with its own pointers")
    p.add_argument("--bandk-caps", default="32,4", help="Band-k caps 'sr,ssr'")
    p.add_argument("--batch-only", action="store_true",
                   help="run only the batched section (profiling); prints {'batch': ...}")
    p.add_argument("--fem", action="store_true",
                   help="run only the FEM-like 160^3 SpMV; prints {'fem': ...}")
    p.add_argument("--irregular", action="store_true",
                   help="run only the long-row comparison; prints {'irregular': ...}")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    if args.quick:
        args.no_e2e = args.no_graph = args.no_cg = args.no_precision = args.no_fem = True
        args.no_kstudy = args.no_batch = args.no_cpu = True
    world, rank, local = dist_env()
    if args.irregular:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"irregular": run_irregular(args, torch.device("cuda", local))}), flush=True)
        return
    if args.fem:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"fem": run_fem(args, torch.device("cuda", local))}), flush=True)
        return
    if args.batch_only:
        import torch
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        peak, _ = measured_peaks()
        out = run_batch(args, dev, torch.cuda.current_stream(dev), peak)
        print(json.dumps({"batch": out}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
