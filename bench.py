#!/usr/bin/env python
"""Benchmark of the CSR-k SpMV hot path on GB300.

Workload (one "step"): y = A x on two 128^3 stencil matrices, 7-point (n = 2,097,152,
nnz = 14,581,760) and 27-point (nnz = 55,742,968); FP64 values diagonally dominant with
off-diagonals U[-1,0), int32 indices; the input rows/columns carry a random symmetric
permutation (seed 3) that the CSR-k reorder (RCM) undoes; CSR-3 sizes and launch shape
from the library's autotuner; x ~ U[-1,1] (seed 2).  Each step runs, per matrix: permute
x into the reordered numbering, then the CSR-3 kernel storing y in the input numbering
(fused unpermute) -- the whole device path of a natural-numbering csrk_spmv call.  Inputs are resident in HBM
and each step's working set (~930 MB) exceeds the 129 MB L2, so no flush is needed.

Metric: GFLOP/s (2 flops per stored nonzero per SpMV), whole job over all ranks.
Roofline: HBM bytes of the dominant kernel (the 27-point CSR-3 launch) per launch over its
mean CUDA-event duration, against the measured copy bandwidth.

--impl reference times the FP64 CPU oracle (single thread, plain CSR loop) on the host
cores on a bounded sample of the same workload.

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
WORKLOAD = ("128^3 7-point and 27-point random diagonally dominant stencils (FP64 values, int32 "
            "indices), rows/columns under a random symmetric permutation; y = A x per matrix per step, "
            "x and y in the input numbering")
SR, SSR = 32, 8
MATRICES = (("stencil7", 7), ("stencil27", 27))

# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by (matrix,
# dtype, kernel number) and valid only for the kernel source it was taken on.  Each entry
# is a 96^3 capture (profiles/csr3_tma_27pt_96cubed_f64.md: 299.20 MB, kernel 0;
# profiles/csr3_tma_k4_27pt_96cubed_f64.md: 252.25 MB, kernel 4) scaled to 128^3 by
# nonzeros.
NCU_TRAFFIC = {
    ("stencil27", "f64", 0): {"bytes": 712_940_980, "kernel_hash": "871b5d682a86"},
    ("stencil27", "f64", 4): {"bytes": 601_073_144, "kernel_hash": "150e04d362cd"},
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


def alg_bytes_spmv(n, nnz, nsr, nssr, val_bytes=8, x_bytes=8, fused_unpermute=True, col_bytes=4):
    # every stored value and column index (4 bytes, or a 2-byte offset with kernel 4),
    # rowptr, sr_ptr, the 32-byte SSR descriptors, x read once and y written once
    # (beta = 0), and the permutation read once when the kernel stores y in the input
    # numbering
    return ((val_bytes + col_bytes) * nnz + 4 * (n + 1) + 4 * (nsr + 1) + 32 * nssr + x_bytes * n + x_bytes * n
            + (4 * n if fused_unpermute else 0))


def col_bytes_of(cfg):
    return 2 if cfg.get("kernel") == 4 else 4


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


def cpu_oracle_gflops(mats, seconds):
    """The FP64 oracle (plain C row loop, one thread) on whole matrices, repeated until
    `seconds` have passed."""
    from oracle import spmv as ospmv
    x = {}
    flops = 0.0
    t0 = time.perf_counter()
    reps = 0
    while True:
        for name, a in mats:
            if name not in x:
                x[name] = synth.uniform_vector(a.n, 2)
            ospmv.csr_spmv(a.n, a.rowptr, a.colidx, a.vals, x[name])
            flops += 2.0 * a.nnz
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return flops / dt / 1e9, f"{reps} full SpMV pass(es) over both 128^3 matrices in {dt:.1f} s"


# ------------------------------------------------------------------ our arm
def run_ours(args, world, rank, local):
    import ctypes

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
        state.append(dict(name=name, a=a, h=h, info=inf, x=x, xp=xp, yp=yp, y=y,
                          cfg=csrk.tuned_config(h), tune_s=t_tune, order_s=t_order))

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
    # correctness guard on sampled rows before timing
    from oracle import spmv as ospmv
    for s in state:
        rows = np.random.default_rng(1).integers(0, s["a"].n, 2000)
        ref = ospmv.csr_spmv_rows(s["a"].rowptr, s["a"].colidx, s["a"].vals, s["x"].cpu().numpy(), rows)
        scale = ospmv.abs_row_scale(s["a"].rowptr, s["a"].colidx, s["a"].vals, s["x"].cpu().numpy(), rows=rows)
        got = s["y"].cpu().numpy()[rows]
        tol = 1e-12 if args.dtype == "f64" else 2.0 ** -8
        if np.any(np.abs(got - ref) > tol * scale):
            raise RuntimeError(f"{s['name']}: result check failed before timing")

    K = args.steps
    events = [[[torch.cuda.Event(enable_timing=True) for _ in range(K)] for _ in range(3)] for _ in state]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    dom = max(range(len(state)), key=lambda j: statistics.mean(kern_ms[j]))
    sd = state[dom]
    inf = sd["info"]
    abytes = alg_bytes_spmv(inf["n"], inf["nnz"], inf["nsr"], inf["nssr"], vb, col_bytes=col_bytes_of(sd["cfg"]))
    kmean = statistics.mean(kern_ms[dom])
    achieved = abytes / (kmean * 1e-3) / 1e9
    khash = kernel_source_hash()
    tr = NCU_TRAFFIC.get((sd["name"], args.dtype, sd["cfg"]["kernel"]))
    traffic = tr["bytes"] if tr and tr["kernel_hash"] == khash else None

    per_matrix = {}
    for j, s in enumerate(state):
        inf = s["info"]
        km = statistics.mean(kern_ms[j])
        b = alg_bytes_spmv(inf["n"], inf["nnz"], inf["nsr"], inf["nssr"], vb, col_bytes=col_bytes_of(s["cfg"]))
        per_matrix[s["name"]] = {"n": inf["n"], "nnz": inf["nnz"], "kernel_us": round(km * 1e3, 2),
                                 "kernel_min_us": round(min(kern_ms[j]) * 1e3, 2),
                                 "kernel_gflops": round(2.0 * inf["nnz"] / (km * 1e-3) / 1e9, 1),
                                 "kernel_gbs": round(b / (km * 1e-3) / 1e9, 1),
                                 "kernel_frac_of_peak": round(b / (km * 1e-3) / 1e9 / peak, 3),
                                 "permute_us": round(statistics.mean(perm_ms[j]) * 1e3, 2),
                                 "sr": inf["sr"], "ssr": inf["ssr"], "nsr": inf["nsr"], "nssr": inf["nssr"],
                                 "config": s["cfg"],
                                 "setup_s": round(s["tune_s"], 2), "order_s": round(s["order_s"], 2)}

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
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(E):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        e2e = {"value": round(whole_job_rate(world, E * flops_step, ems) / 1e9, 2), "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(sum(8 * s["a"].n for s in state)),
               "d2h_bytes_per_step": int(sum(8 * s["a"].n for s in state))}

    # conjugate gradients to rtol 1e-10 on the 27-point matrix: FP64 against mixed precision
    cg = None
    if not args.no_cg:
        s27 = state[-1]
        b = torch.tensor(synth.uniform_vector(s27["a"].n, 5), dtype=torch.float64, device=dev)
        xs = torch.empty_like(b)
        cg = {"matrix": s27["name"], "rtol": 1e-10, "replace_every": 20, "runs": {}}
        for inner, restart in (("f64", 0), ("f32", 0), ("bf16", 1)):
            csrk.cg(s27["h"], b, xs, 1e-10, 5000, inner, 20, restart)     # capture the graphs
            torch.cuda.synchronize()
            times = []
            for rep in range(3):
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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

    batch = None
    if not args.no_batch:
        batch = run_batch(args, dev, stream, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        g, sample = cpu_oracle_gflops(mats, args.cpu_seconds)
        cpu = {"value": round(g, 3), "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample}

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
            "config": {"workload": WORKLOAD,
                       "method": "CSR-3 sizes and launch shape from the library autotuner; per matrix "
                                 "permute x, then the CSR-3 kernel storing y in the input numbering",
                       "sizes": args.sizes, "ordering": args.ordering if args.ordering == "rcm" else
                       f"bandk {args.bandk_caps}", "l2": "inputs larger than L2 (~930 MB per step vs 129 MB)",
                       "parallelism": f"replicas x{world}", "per_matrix": per_matrix},
            "roofline": {"bound": "hbm", "kernel": f"csr3 {state[dom]['name']}",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "alg_bytes_per_launch": int(abytes), "peak_kind": peak_kind,
                         "kernel_hash": khash,
                         # the same launch against GB300's FP64 FMA rate (one FMA per nonzero):
                         # the SpMV is co-bound by HBM and the FP64 pipe
                         "fp64": {"achieved_gflops": round(2.0 * sd["info"]["nnz"] / (kmean * 1e-3) / 1e9, 1),
                                  "peak_gflops": FP64_NOMINAL_GFLOPS, "peak_kind": "nominal",
                                  "frac": round(2.0 * sd["info"]["nnz"] / (kmean * 1e-3) / 1e9
                                                / FP64_NOMINAL_GFLOPS, 4)}},
            "e2e": e2e,
            "cg": cg,
            "batch": batch,
            "gpu_launches": K * 2 * len(state),   # per matrix: permute x, CSR-3 kernel (+ fused unpermute)
            "clocks": clocks,
            "cpu_baseline": cpu,
            "wall_s_timed": round(wall, 3),
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


def run_fem(args, dev):
    """The FEM-like SPD matrix on 160^3 jittered points (n = 4,096,000, ~61 M nonzeros,
    12-18 neighbours per row, random labels): natural-numbering SpMV (permute x, CSR-3
    kernel with the fused unpermute), autotuned, kernel time with CUDA events and the same
    algorithmic-byte roofline as the stencils."""
    import torch
    from paper_2203_05096_gb300 import csrk
    t0 = time.perf_counter()
    a = synth.fem_like(160, 4)
    gen_s = time.perf_counter() - t0
    x = torch.tensor(synth.uniform_vector(a.n, 2), dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h, "rcm", want_perm=False)
    csrk.set_sizes(h, 0, 0)
    for _ in range(5):
        csrk.spmv(h, 1.0, x, 0.0, y)
    torch.cuda.synchronize()
    reps = max(20, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    e0.record(stream)
    for _ in range(reps):
        csrk.spmv(h, 1.0, xp, 0.0, y, csrk.X_PERMUTED)
    e1.record(stream)
    torch.cuda.synchronize()
    kus = e0.elapsed_time(e1) / reps * 1e3
    ab = alg_bytes_spmv(inf["n"], inf["nnz"], inf["nsr"], inf["nssr"], 8, col_bytes=col_bytes_of(cfg))
    out = {"workload": "FEM-like SPD, 160^3 jittered points, 12-18 neighbours per row, random labels, FP64",
           "n": int(a.n), "nnz": int(a.nnz), "generate_s": round(gen_s, 1), "config": cfg,
           "sr": inf["sr"], "ssr": inf["ssr"], "call_us": round(us, 2),
           "call_gflops": round(2.0 * a.nnz / (us * 1e-6) / 1e9, 1), "kernel_us": round(kus, 2),
           "kernel_gflops": round(2.0 * a.nnz / (kus * 1e-6) / 1e9, 1),
           "kernel_alg_bytes": int(ab), "kernel_gbs": round(ab / (kus * 1e-6) / 1e9, 1),
           "kernel_frac_of_peak": round(ab / (kus * 1e-6) / 1e9 / peak, 3), "peak_kind": peak_kind}
    csrk.destroy(h)
    return out


# ------------------------------------------------------------------ reference arm
def run_reference(args, world, rank, local):
    """The FP64 CPU oracle as it stands, on the host cores, each step a bounded block of
    rows of both matrices (rotating through the matrix)."""
    if rank != 0:
        return
    from oracle import spmv as ospmv
    mats = build_matrices(args.side, args.only)
    xs = [synth.uniform_vector(a.n, 2) for _, a in mats]
    budget = max(0.005, min(0.5, 60.0 / max(1, args.steps + args.warmup)))
    # calibrate rows per block on the densest matrix
    a27 = mats[-1][1]
    probe = np.arange(0, 20000, dtype=np.int64)
    t0 = time.perf_counter()
    ospmv.csr_spmv_rows(a27.rowptr, a27.colidx, a27.vals, xs[1], probe)
    per_row = (time.perf_counter() - t0) / probe.size
    rows_per_block = max(1000, int(budget / 2 / max(per_row, 1e-9)))
    cursor = [0, 0]

    def step():
        fl = 0.0
        for j, (_, a) in enumerate(mats):
            b = cursor[j]
            e = min(a.n, b + rows_per_block)
            rows = np.arange(b, e, dtype=np.int64)
            ospmv.csr_spmv_rows(a.rowptr, a.colidx, a.vals, xs[j], rows)
            fl += 2.0 * float(a.rowptr[e] - a.rowptr[b])
            cursor[j] = 0 if e >= a.n else e
        return fl

    for _ in range(args.warmup):
        step()
    flops = 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flops += step()
    dt = time.perf_counter() - t0
    value = flops / dt / 1e9
    sample = f"{rows_per_block} rows of each matrix per step, {args.steps} steps, {dt:.1f} s"
    line = {
        "impl": "reference",
        "metric": "SpMV GFLOP/s (CSR-3, 128^3 7-point + 27-point stencils, FP64)",
        "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "method": "FP64 CPU oracle: plain CSR loop over the matrices in the input numbering"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
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
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cg", action="store_true")
    p.add_argument("--no-batch", action="store_true")
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
