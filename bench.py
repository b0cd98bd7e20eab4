"""Benchmark of the repeated-block SpMM hot path on one GB300 (or N independent replicas).

Workload: the channel-flow-shaped staggered grid 192 x 128 x 96 (n = 2,359,296 cells,
7,059,456 faces; periodic x and z, walls in y refined by tanh with factor 1.5).  One step
applies the discrete operators as SpMM over k right-hand sides, in FP64 and in FP32:
    Laplacian L (k = 3, velocity components), gradient G (k = 3), divergence M (k = 1).
metric value = effective GFLOP/s of the step: sum over its SpMMs of 2 nnz k, divided by the
device time of the step.  Beside it the same run reports, each timed with CUDA events:
  * spmm: per operator / dtype / k: time, GFLOP/s, algorithmic GB/s, fraction of the
    measured HBM copy bandwidth, and the k-sweep of the Laplacian (k = 1 .. 32);
  * poisson: ms to a 1e-10 true relative residual, FP64 Jacobi-CG vs FP32-inner FP64
    refinement, on the compatible right-hand sides b = M u (k = 3 flow states);
  * roofline of the dominant kernel, e2e through host buffers, the oracle on the host
    cores (cpu_baseline), and the SM clocks sampled during the timed region.

--impl reference times the CPU oracle (plain FP64 scipy, one core) on the same workload.
Under torchrun (N > 1) every rank runs an independent replica (the path does not shard
across GPUs here); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SpMM effective GFLOP/s & HBM GB/s vs k; Poisson solve ms to 1e-10 residual vs FP64 CG"
WORKLOAD = "channel 192x128x96 staggered FVM: L,G SpMM k=3 + M SpMM k=1, FP64 and FP32"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 FMA throughput of a GB300: the nominal dense FP64 rate (1.25 TFLOP/s).  The path's
# FP64 SpMM with k >= 2 is bound by it rather than by HBM.
FP64_PEAK_TFLOPS = 1.25


# DRAM traffic (read + write) per launch of the dominant kernel, from one ncu capture of the
# timed step, valid only for the SpMM sources it was taken with: the fingerprint of those
# sources is checked at run time, and traffic is null (not measured for this build) when they
# have changed.
SPMM_SOURCES = ['spmm_impl.cuh', 'spmm_kernels.cuh', 'spmm_f64.cu', 'spmm_f32.cu', 'spmm_tma.cuh', 'common.cuh', 'tma.cuh', 'spmm.cu']
TRAFFIC = {"L-f64-k3": (264_993_792 + 42_707_200, "92f1acc610ff2014")}


def spmm_fingerprint():
    import hashlib

    h = hashlib.sha256()
    for f in SPMM_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2508_06710_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel_label):
    t = TRAFFIC.get(kernel_label)
    return t[0] if t and t[1] == spmm_fingerprint() else None


def spmm_bytes(nnz, n_r, n_c, k, s):
    """Algorithmic bytes of one CSR SpMM: matrix once (value + index), row pointers, X read once, Y written."""
    return nnz * (s + 4) + 4 * (n_r + 1) + s * k * (n_r + n_c)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def face_starts(g):
    """First rows of the x-, y- and z-face blocks of the gradient of grid g (faces numbered by
    direction; a bounded axis has n - 1 interior faces, a periodic one n)."""
    n = [a.n for a in g.axes]
    counts = []
    for d in range(3):
        c = n[d] if g.axes[d].periodic else n[d] - 1
        for e in range(3):
            if e != d:
                c *= n[e]
        counts.append(c)
    return [0, counts[0], counts[0] + counts[1]]


def build_ops(rb, torch, dev):
    """Operators of the channel workload, assembled on the device by the library."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    nodes, per = rb.grid_nodes(g, dev)
    ops = {}
    for name, kind, k in (("L", rb.RB_FVM_LAPLACIAN, 3), ("G", rb.RB_FVM_GRADIENT, 3), ("M", rb.RB_FVM_DIVERGENCE, 1)):
        rp, ci, va, nc = rb.fvm_assemble(nodes, per, kind)
        for dt in ("f64", "f32"):
            ops[(name, dt)] = (rb.Operator(rp, ci, va, nc, dtype=dt, k_max=32), k)
            ops[(name + "-sell", dt)] = (rb.Operator(rp, ci, va, nc, dtype=dt, fmt="sell", k_max=32), k)
        ops[(name, "df64")] = (rb.Operator(rp, ci, va, nc, dtype="df64", k_max=32), k)
        if name == "L":  # the Poisson matrix A = -L, assembled with scale -1
            rp, ci, va, nc = rb.fvm_assemble(nodes, per, kind, scale=-1.0)
            ops[("A", "f64")] = (rb.Operator(rp, ci, va, nc, dtype="f64", k_max=3), 3)
            ops[("A", "f32")] = (rb.Operator(rp, ci, va, nc, dtype="f32", k_max=3), 3)
    torch.cuda.synchronize()
    return g, ops


def run_ours(args, rank, world, local):
    import torch

    import paper_2508_06710_gb300 as rb
    from paper_2508_06710_gb300 import build as rbbuild

    rbbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    torch.manual_seed(2508_06710 + rank)  # the sweeps' N(0,1) blocks (torch.randn) are seeded too
    stream = torch.cuda.current_stream()
    g, ops = build_ops(rb, torch, dev)
    hbm, hbm_src = peaks()
    # inputs (seeded, resident in HBM before timing)
    step_items = []  # (label, op, X, Y, k, dtype)
    for name in ("L", "G", "M"):
        for dt in ("f64", "f32"):
            op, k = ops[(name, dt)]
            tdt = torch.float64 if dt == "f64" else torch.float32
            X = torch.as_tensor(W.normal((op.n_cols, k), W.seed_for(2, k, salt=len(step_items))), device=dev).to(tdt)
            Y = torch.empty((op.n_rows, k), dtype=tdt, device=dev)
            op.tune(X, Y)
            step_items.append((f"{name}-{dt}-k{k}", op, X, Y, k, dt))
    flops_step = sum(2 * it[1].nnz * it[4] for it in step_items)

    # Each kernel's duration: the interval between the timing events on either side of it.
    # Adjacent kernels share the event between them (7 events a step, not 12): every timing
    # event holds the stream for a few microseconds.
    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        for i, (label, op, X, Y, k, _) in enumerate(step_items):
            if args.nvtx:
                torch.cuda.nvtx.range_push(label)
            op.spmm(X, Y)
            if args.nvtx:
                torch.cuda.nvtx.range_pop()
            if evs is not None:
                evs[i + 1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    per_kernel = [[torch.cuda.Event(enable_timing=True) for _ in range(len(step_items) + 1)]
                  for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if args.nvtx:
        torch.cuda.nvtx.range_push("timed_step")
    t0.record(stream)
    for s in range(args.steps):
        step(per_kernel[s])
    t1.record(stream)
    if args.nvtx:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(torch, t0.elapsed_time(t1), world, dev)
    ms_step = ms_total / args.steps
    value = world * flops_step / (ms_step * 1e-3) / 1e9
    # per kernel: average device time over the timed steps
    kern = []
    for i, (label, op, X, Y, k, dt) in enumerate(step_items):
        ts = [per_kernel[s][i].elapsed_time(per_kernel[s][i + 1]) for s in range(args.steps)]
        ms = sum(ts) / len(ts)
        s_b = 8 if dt == "f64" else 4
        by = spmm_bytes(op.nnz, op.n_rows, op.n_cols, k, s_b)
        fl = 2 * op.nnz * k
        kern.append({"kernel": label, "ms": ms, "gflops": fl / ms / 1e6, "gbs": by / ms / 1e6,
                     "frac_hbm": by / ms / 1e6 / hbm, "bytes": by, "flops": fl,
                     "fp64_frac": (fl / ms / 1e9 / FP64_PEAK_TFLOPS) if dt == "f64" else None,
                     "schedule": op.schedule(X, Y)})
    # the ceiling a kernel of this size can reach: a device copy moving the same bytes
    for r in kern:
        src = torch.empty(r["bytes"] // 8, dtype=torch.float32, device=dev)
        dst = torch.empty_like(src)
        r["copy_frac"] = graph_ms(torch, lambda: dst.copy_(src)) / r["ms"]
        del src, dst
    dom = max(kern, key=lambda r: r["ms"])
    overlap = overlapped_step(torch, args, step_items, stream, flops_step, ms_step, world, dev)
    # the FMA roofs measured on this GPU now (the library's rb_fma_peak), beside the nominal one
    fma_meas = {"f64_tflops": rb.fma_peak("f64"), "f32_tflops": rb.fma_peak("f32")}
    if dom["kernel"].split("-")[1] == "f64" and dom["flops"] / (FP64_PEAK_TFLOPS * 1e12) > dom["bytes"] / (hbm * 1e9):
        roof = {"bound": "alu", "achieved": dom["gflops"] / 1e3, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": dom["gflops"] / 1e3 / FP64_PEAK_TFLOPS,
                "traffic": args.traffic if args.traffic else measured_traffic(dom["kernel"]),
                "kernel": dom["kernel"],
                "peak_source": "nominal FP64 FMA rate of GB300: 152 SMs x 2 FP64 FMAs per clock x 2 flops x 2.07 GHz",
                "peak_measured": fma_meas["f64_tflops"], "frac_of_measured": dom["gflops"] / 1e3 / fma_meas["f64_tflops"],
                "hbm_gbs": dom["gbs"], "hbm_frac_of_measured": dom["frac_hbm"]}
    else:
        roof = {"bound": "hbm", "achieved": dom["gbs"], "peak": hbm, "unit": "GB/s", "frac": dom["frac_hbm"],
                "traffic": args.traffic if args.traffic else measured_traffic(dom["kernel"]),
                "kernel": dom["kernel"], "peak_source": hbm_src}
    out = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_cells": g.n_cells, "k": {"L": 3, "G": 3, "M": 1},
                      "l2": "inputs larger than L2: every SpMM streams >= 160 MB", "parallelism": "replicas"},
           "roofline": roof, "fma_peaks_measured": fma_meas, "kernels": kern,
           "gpu_launches": len(step_items) * args.steps, "clocks": clk, "overlapped_step": overlap}
    if rank == 0 and not args.quick:
        out["e2e"] = e2e(args, torch, step_items, stream, dev, flops_step)
        out["ksweep"] = k_sweep(torch, rb, ops, dev, hbm)
        out["ksweep_stencil"] = k_sweep_stencil(torch, rb, g, dev, hbm)
        out["step_variants"] = step_variants(torch, rb, ops, g, dev, hbm)
        out["poisson"] = poisson(torch, rb, ops, g, dev)
        out["multigrid"] = multigrid(torch, rb, g, dev, out["poisson"])
        out["operator_build"] = operator_build(torch, rb, g, dev)
        out["blas1"] = blas1(torch, rb, dev, g.n_cells, hbm)
        out["stencils"] = stencils(torch, rb, dev, hbm)
        out["refine"] = refine_maps(torch, rb, dev, hbm)
        out["projection"] = projection(torch, rb, dev)
        out["refinement_run"] = refinement_run(torch, rb, dev)
        del ops, step_items
        torch.cuda.empty_cache()
        out["batch"] = batch_bench(torch, rb, dev)
        out["extruded"] = extruded_bench(torch, rb, dev, hbm)
        out["rbc_spmm"] = rbc_spmm(torch, rb, dev, hbm)
        k8 = [r for r in out["ksweep"] if r["format"] == "csr" and r["k"] == 8]
        out["paper_context"] = dict(PAPER_CONTEXT, this_gpu_spmm_speedup_vs_k_spmv_k8={r["dtype"]: r["speedup_vs_k_spmv"]
                                                                                     for r in k8})
        if not args.no_guess:
            torch.cuda.empty_cache()
            out["learned_guess"] = learned_guess(torch, rb, dev, args)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(g)
    return out


def operator_build(torch, rb, g, dev):
    """Device assembly of L, G, M on the channel grid (events, median of 5)."""
    nodes, per = rb.grid_nodes(g, dev)
    res = {}
    for name, kind in (("L", rb.RB_FVM_LAPLACIAN), ("G", rb.RB_FVM_GRADIENT), ("M", rb.RB_FVM_DIVERGENCE)):
        nr, nc, nnz = rb.fvm_csr_size(nodes, per, kind)
        rp = torch.empty(nr + 1, dtype=torch.int32, device=dev)
        ci = torch.empty(nnz, dtype=torch.int32, device=dev)
        va = torch.empty(nnz, dtype=torch.float64, device=dev)
        gd = rb._grid_desc(nodes, per)
        import ctypes as C

        def run():
            rb._check(rb.lib().rb_fvm_assemble(C.byref(gd), kind, 1.0, rb._ptr(rp), rb._ptr(ci), rb._ptr(va),
                                               rb._stream()), "rb_fvm_assemble")

        ms = time_events(torch, run, 5)
        res[name] = {"ms": ms, "nnz": nnz, "gbs_written": (nnz * 12 + 4 * (nr + 1)) / ms / 1e6}
    return res


STENCIL_N = 160  # the fine mesh on which Sec. 4.1 compares the 7p, 13p and 27p patterns


def stencils(torch, rb, dev, hbm):
    """SpMM on the 7p (FVM), 13p and 27p Laplacians of the uniform periodic 160^3 grid (Sec. 4.1's
    denser patterns), FP64 and FP32, k = 1, 2, 4, 8 (tuned; events, median of 10): GFLOP/s,
    algorithmic GB/s and the speed-up over k SpMVs, k t_1 / t_k; and the device assembly of
    each 13p / 27p CSR (events, median of 5)."""
    import ctypes as C

    n, h = STENCIL_N, 1.0 / STENCIL_N
    cells = n ** 3
    res = {"grid": f"periodic {n}^3", "n": cells, "spmm": [], "assembly": {}}
    for name in ("7p", "13p", "27p"):
        if name == "7p":
            nodes, per = rb.grid_nodes(W.unit_periodic_grid(n), dev)
            rp, ci, va, _ = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
        else:
            kind = rb.RB_STENCIL_13P if name == "13p" else rb.RB_STENCIL_27P
            rp, ci, va, _ = rb.stencil_assemble((n, n, n), (h, h, h), kind, device=dev)
            narr, harr = (C.c_int32 * 3)(n, n, n), (C.c_double * 3)(h, h, h)

            def run():
                rb._check(rb.lib().rb_stencil_assemble(narr, harr, kind, 1.0, rb._ptr(rp), rb._ptr(ci), rb._ptr(va),
                                                       rb._stream()), "rb_stencil_assemble")

            ms = time_events(torch, run, 5)
            res["assembly"][name] = {"ms": ms, "nnz": ci.numel(), "gbs_written": (ci.numel() * 12 + 4 * (cells + 1)) / ms / 1e6}
        for dt in ("f64", "f32"):
            op = rb.Operator(rp, ci, va, cells, dtype=dt, k_max=8)
            tdt = torch.float64 if dt == "f64" else torch.float32
            s_b = 8 if dt == "f64" else 4
            base = None
            for k in (1, 2, 4, 8):
                X = torch.randn((cells, k), dtype=tdt, device=dev)
                Y = torch.empty((cells, k), dtype=tdt, device=dev)
                op.tune(X, Y)
                by = spmm_bytes(op.nnz, cells, cells, k, s_b)
                ms = spmm_ms(torch, op, X, Y, by)
                base = ms if k == 1 else base
                res["spmm"].append({"stencil": name, "dtype": dt, "k": k, "nnz": op.nnz, "ms": ms,
                                    "gflops": 2 * op.nnz * k / ms / 1e6, "gbs": by / ms / 1e6, "frac_hbm": by / ms / 1e6 / hbm,
                                    "ai_flop_per_byte": 2 * op.nnz * k / by, "speedup_vs_k_spmv": k * base / ms,
                                    "schedule": op.schedule(X, Y)})
                del X, Y
            del op
        del rp, ci, va
        torch.cuda.empty_cache()
    return res


def refine_maps(torch, rb, dev, hbm):
    """Inline mesh refinement (Sec. 3.3): the k states of the 96 x 64 x 48 channel mapped onto
    192 x 128 x 96 by the prolongation P (8 entries per fine row) and back by the restriction R,
    FP64 and FP32, k = 1, 3, 4, 8 (tuned; events, median of 10); and the device assembly of P
    and R (events, median of 5)."""
    import ctypes as C

    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    nodes, per = rb.grid_nodes(g, dev)
    res = {"fine": "channel 192x128x96", "coarse": "channel 96x64x48", "spmm": [], "assembly": {}}
    for name, kind in (("prolong", rb.RB_REFINE_PROLONG), ("restrict", rb.RB_REFINE_RESTRICT)):
        rp, ci, va, nc = rb.refine_assemble(nodes, per, kind)
        gd = rb._grid_desc(nodes, per)

        def run():
            rb._check(rb.lib().rb_refine_assemble(C.byref(gd), kind, rb._ptr(rp), rb._ptr(ci), rb._ptr(va), rb._stream()),
                      "rb_refine_assemble")

        ms = time_events(torch, run, 5)
        nr = rp.numel() - 1
        res["assembly"][name] = {"ms": ms, "nnz": ci.numel(), "gbs_written": (ci.numel() * 12 + 4 * (nr + 1)) / ms / 1e6}
        for dt in ("f64", "f32"):
            op = rb.Operator(rp, ci, va, nc, dtype=dt, k_max=8)
            tdt = torch.float64 if dt == "f64" else torch.float32
            s_b = 8 if dt == "f64" else 4
            for k in (1, 3, 4, 8):
                X = torch.randn((nc, k), dtype=tdt, device=dev)
                Y = torch.empty((nr, k), dtype=tdt, device=dev)
                op.tune(X, Y)
                by = spmm_bytes(op.nnz, nr, nc, k, s_b)
                ms = spmm_ms(torch, op, X, Y, by)
                res["spmm"].append({"map": name, "dtype": dt, "k": k, "ms": ms, "gflops": 2 * op.nnz * k / ms / 1e6,
                                    "gbs": by / ms / 1e6, "frac_hbm": by / ms / 1e6 / hbm, "schedule": op.schedule(X, Y)})
                del X, Y
            del op
        del rp, ci, va
    torch.cuda.empty_cache()
    return res


FLOW_N = 128  # the periodic 128^3 box of the batched systems, here in 2 pi units


def projection(torch, rb, dev):
    """Heun RK3 projection steps of Eq. (ns) on m = 1, 2, 4, 8 stacked flow states (the
    paper's ensemble of Sec. 3.1) in the periodic 2 pi box of 128^3 cells: Taylor-Green
    vortices of amplitude 1 + 0.1 s plus seeded noise of 0.01, nu = 0.01, dt = 0.01, the
    Poisson solves by the FP32-inner refinement to 1e-10 from the previous step's pressure.
    One warm-up step, then three timed (host clock around synchronised steps: every solve
    synchronises to read its report).  Reports ms per step, the Poisson share and the speed-up
    of one m-state step over m single-state steps (the iteration speed-up of Eq. (pmite)), with
    the pressure solved by the multigrid CG and by the Jacobi-preconditioned CG."""
    import math

    from paper_2508_06710_gb300.flow_step import ProjectionStep

    n, nu, dt = FLOW_N, 0.01, 0.01
    L = 2 * math.pi
    nodes = [torch.linspace(0.0, L, n + 1, dtype=torch.float64, device=dev) for _ in range(3)]
    cells = n ** 3
    h = L / n
    c = (torch.arange(n, dtype=torch.float64, device=dev) + 0.5) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    su, sv = (torch.sin(x) * torch.cos(y)).reshape(-1), (-torch.cos(x) * torch.sin(y)).reshape(-1)
    res = {"grid": f"periodic {n}^3, 2 pi", "nu": nu, "dt": dt, "steps": 3, "states": []}
    for solver in ("mg", "jacobi"):
        _projection_runs(torch, res, nodes, n, cells, nu, dt, su, sv, solver, dev)
    return res


def _projection_runs(torch, res, nodes, n, cells, nu, dt, su, sv, solver, dev):
    from paper_2508_06710_gb300.flow_step import ProjectionStep

    base = None
    for m in (1, 2, 4, 8):
        stepper = ProjectionStep(torch, nodes, m, nu, dt, mixed=2, solver=solver)
        u = torch.as_tensor(0.01 * W.normal((cells, 3 * m), 1900 + m), device=dev)
        for s in range(m):
            u[:, s] += (1 + 0.1 * s) * su
            u[:, m + s] += (1 + 0.1 * s) * sv
        us = torch.zeros((3 * cells, m), dtype=torch.float64, device=dev)
        stepper.step(u, us)
        torch.cuda.synchronize()
        stepper.poisson_ms, stepper.iters = 0.0, []
        t0 = time.perf_counter()
        for _ in range(3):
            stepper.step(u, us)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / 3
        base = ms if m == 1 else base
        res["states"].append({"solver": solver, "m": m, "ms_per_step": ms, "ms_per_state_step": ms / m,
                              "poisson_share": stepper.poisson_ms / 3 / ms, "solve_iters": stepper.iters,
                              "speedup_vs_m_single": m * base / ms})
        del stepper, u, us
        torch.cuda.empty_cache()


def refinement_run(torch, rb, dev, steps=3):
    """Inline mesh refinement (Sec. 3.3) over a time-step sequence: m = 1, 2, 4, 8 stacked flow
    states developed on the 64^3 periodic 2 pi box (dt = 0.02), mapped onto 128^3 (trilinear P
    over the 3 m columns, then a projection) and continued there (dt = 0.01); Taylor-Green
    vortices of amplitude 1 + 0.1 s plus seeded noise of 0.01, nu = 0.01; pressure solves by
    the multigrid CG (FP32 cycle inside FP64 refinement) to 1e-10 from the previous pressure.
    Per m: ms per coarse step and per fine step (host clock around synchronised steps, after
    one untimed step on each grid), the mapping's ms, the mesh pace ratio delta_m = f^C / f^F
    with f = (ms per step) / dt (Sec. 3.3's simulation pace), the fine grid's iteration
    speed-up m t_1 / t_m, and the whole-simulation speed-up of Eq. (speedup1) at the paper's
    beta = 10, gamma = 15 beside the single-mesh one (gamma = 0)."""
    import math

    from paper_2508_06710_gb300.flow_step import RefinedEnsemble

    nf, nu, dtf = 2 * 64, 0.01, 0.01
    L = 2 * math.pi
    nodes = [torch.linspace(0.0, L, nf + 1, dtype=torch.float64, device=dev) for _ in range(3)]
    nc = nf // 2
    h = L / nc
    c = (torch.arange(nc, dtype=torch.float64, device=dev) + 0.5) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    su, sv = (torch.sin(x) * torch.cos(y)).reshape(-1), (-torch.cos(x) * torch.sin(y)).reshape(-1)
    res = {"coarse": f"periodic {nc}^3", "fine": f"periodic {nf}^3", "dt_coarse": 2 * dtf, "dt_fine": dtf, "nu": nu,
           "steps": steps, "states": []}
    base = None
    for m in (1, 2, 4, 8):
        run = RefinedEnsemble(torch, nodes, m, nu, dtf, mixed=2, solver="mg")
        u = torch.as_tensor(0.01 * W.normal((nc ** 3, 3 * m), 2900 + m), device=dev)
        for s in range(m):
            u[:, s] += (1 + 0.1 * s) * su
            u[:, m + s] += (1 + 0.1 * s) * sv
        us = torch.zeros((3 * nc ** 3, m), dtype=torch.float64, device=dev)
        run.coarse.step(u, us)  # untimed: records the solver's graphs
        uf, usf, t = run.run(u, us, steps, 0)
        run.fine.step(uf, usf)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            run.fine.step(uf, usf)
        torch.cuda.synchronize()
        ms_f = (time.perf_counter() - t0) * 1e3 / steps
        ms_c = t["coarse_ms"] / steps
        f_c, f_f = ms_c / (2 * dtf), ms_f / dtf
        rec = {"m": m, "ms_per_coarse_step": ms_c, "ms_per_fine_step": ms_f, "map_ms": t["map_ms"],
               "delta_m": f_c / f_f, "Pi_m": f_f / f_c, "fine_solve_iters": run.fine.iters[-3:]}
        if m == 1:
            base = rec
        rec["fine_iteration_speedup"] = m * base["ms_per_fine_step"] / ms_f
        beta, gamma = 10.0, 15.0
        d1, dm = base["delta_m"], rec["delta_m"]
        # Eq. (speedup1): (1 + d1 g + (1 + g) b) / (m (dm g + 1) + (1 + g) b) * m f_1^F / f_m^F
        rec["simulation_speedup_refined"] = ((1 + d1 * gamma + (1 + gamma) * beta) / (m * (dm * gamma + 1) + (1 + gamma) * beta)
                                             * rec["fine_iteration_speedup"])
        rec["simulation_speedup_single_mesh"] = (1 + beta) / (m + beta) * rec["fine_iteration_speedup"]
        res["states"].append(rec)
        del run, u, us, uf, usf
        torch.cuda.empty_cache()
    return res


def overlapped_step(torch, args, step_items, stream, flops_step, ms_serial, world, dev):
    """The same K steps issued the way an application would: the six SpMMs are independent, so
    the FP64 ones (bound by the FP64 pipe) go to one stream and the FP32 ones (bound by HBM) to
    a second, joined at the end of each step, and their kernels overlap.  Timed by events on the
    first stream around all K steps, with no events between kernels (on a shared GPU a kernel's
    own interval is not its cost).  The timed region above keeps one stream and per-kernel
    events, which the roofline needs; this is the throughput the step reaches without them."""
    side = torch.cuda.Stream()
    f64 = [it for it in step_items if it[5] == "f64"]
    f32 = [it for it in step_items if it[5] == "f32"]

    def step():
        side.wait_stream(stream)
        for a, b in zip(f64, f32):
            a[1].spmm(a[2], a[3], stream=stream)
            b[1].spmm(b[2], b[3], stream=side)
        stream.wait_stream(side)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(torch, t0.elapsed_time(t1), world, dev) / args.steps
    return {"streams": 2, "ms_per_step": ms, "value": world * flops_step / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
            "vs_single_stream": ms_serial / ms, "gpu_launches": len(step_items) * args.steps}


L2_BYTES = 126 * 2 ** 20  # GB300's L2


def spmm_ms(torch, op, X, Y, bytes_per_call, calls=24, reps=5):
    """Device time of one op.spmm on blocks shaped like X, Y, measured without host launch
    latency: a CUDA graph of `calls` SpMMs cycling over enough (X, Y) copies that the blocks of
    consecutive calls exceed twice the L2 (so no call finds its inputs in L2 from the one
    before), replayed `reps` times; the median replay divided by `calls`."""
    copies = max(1, min(calls, -(-2 * L2_BYTES // max(int(bytes_per_call), 1))))
    xs = [X] + [X.clone() for _ in range(copies - 1)]
    ys = [Y] + [torch.empty_like(Y) for _ in range(copies - 1)]
    ms = graph_ms(torch, lambda: [op.spmm(xs[i % copies], ys[i % copies]) for i in range(calls)], calls=1, reps=reps)
    del xs, ys
    return ms / calls


def graph_ms(torch, fn, calls=20, reps=10):
    """Device time per call of `fn`, from replays of a CUDA graph of `calls` calls (launch
    latency amortised: what the kernels themselves take back to back)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(calls):
            fn()
    ms = time_events(torch, g.replay, reps)
    return ms / calls


def blas1(torch, rb, dev, n, hbm):
    """dot, axpy, axty on n x 3 blocks (FP64 and FP32): algorithmic GB/s per call, timed as
    back-to-back kernels (graph replays) and as single eager calls (launch latency included);
    axty with alpha = 1 (the Jacobi product, one multiply per entry) and with another alpha
    (two multiplies per entry, which the FP64 multiply rate bounds before HBM does);
    `copy_frac` compares with a device copy moving the same bytes (the ceiling at this size).
    n is raised to four channel grids (9.4 M rows) so that every operand exceeds L2 even when
    the replays run back to back."""
    n = 4 * n
    res = []
    for dt in (torch.float64, torch.float32):
        k = 3
        X = torch.randn((n, k), dtype=dt, device=dev)
        Y = torch.randn((n, k), dtype=dt, device=dev)
        ones = torch.ones((n, k), dtype=dt, device=dev)
        alpha = torch.full((k,), 1e-3, dtype=torch.float64, device=dev)
        out = torch.empty(k, dtype=torch.float64, device=dev)
        work = torch.empty(rb.lib().rb_dot_workspace_bytes(n, k), dtype=torch.uint8, device=dev)
        s = X.element_size()
        for name, fn, by in (("dot", lambda: rb.dot(X, Y, out=out, work=work), 2 * n * k * s),
                             ("axpy", lambda: rb.axpy(alpha, X, Y), 3 * n * k * s),
                             ("axty", lambda: rb.axty(1.0, ones, Y), 3 * n * k * s),
                             ("axty_scaled", lambda: rb.axty(1.0 + 2.0 ** -20, ones, Y), 3 * n * k * s)):
            ms = graph_ms(torch, fn)
            ms_call = time_events(torch, fn, 10)
            src = torch.empty(by // 8, dtype=torch.float32, device=dev)
            dst = torch.empty_like(src)
            ms_copy = graph_ms(torch, lambda: dst.copy_(src))
            res.append({"op": name, "dtype": "f64" if s == 8 else "f32", "k": k, "ms": ms, "gbs": by / ms / 1e6,
                        "frac_hbm": by / ms / 1e6 / hbm, "copy_frac": ms_copy / ms, "ms_eager_call": ms_call})
            del src, dst
    return res


def rbc_spmm(torch, rb, dev, hbm):
    """The Laplacian SpMM on the Rayleigh-Benard-shaped 128^3 grid (tanh 1.4 walls in z), k = 1, 3, 8."""
    g = W.rbc_grid(W.GUESS_N, 1.4)
    nodes, per = rb.grid_nodes(g, dev)
    rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
    res = []
    for dt in ("f64", "f32"):
        op = rb.Operator(rp, ci, va, nc, dtype=dt, k_max=8)
        tdt = torch.float64 if dt == "f64" else torch.float32
        for k in (1, 3, 8):
            X = torch.randn((op.n_cols, k), dtype=tdt, device=dev)
            Y = torch.empty((op.n_rows, k), dtype=tdt, device=dev)
            op.tune(X, Y)
            by = spmm_bytes(op.nnz, op.n_rows, op.n_cols, k, 8 if dt == "f64" else 4)
            ms = spmm_ms(torch, op, X, Y, by)
            res.append({"dtype": dt, "k": k, "ms": ms, "gflops": 2 * op.nnz * k / ms / 1e6, "gbs": by / ms / 1e6,
                        "frac_hbm": by / ms / 1e6 / hbm})
        op.close()
    return {"grid": f"rbc {W.GUESS_N}^3", "n": g.n_cells, "runs": res}


# The paper's own numbers (CPU, MareNostrum 5 GPP nodes, FP64): context only, not targets.
PAPER_CONTEXT = {
    "hardware": "MareNostrum 5 general-purpose nodes (CPU), FP64, MPI + OpenMP",
    "spmm_speedup_vs_k_spmv_7pt_up_to": 3.0,          # Sec. 5, 7-point stencil, m <= 8
    "spmm_speedup_vs_k_spmv_13pt_27pt_up_to": [3.3, 4.1],
    "poisson_speedup_fine_160cube_m2_m4_m8": [1.498, 1.884, 2.027],  # Table 5, CG + aAMG
    "projection_iteration_speedup_fine_m2_m4_m8": [1.379, 1.630, 1.728],  # Table 5
}


def batch_bench(torch, rb, dev):
    """Uneven systems (64^3 k=8, 128^3 k=1, three 96x64x48 channels k=3): the persistent batched
    refinement under one CUDA graph vs the same refinement per system and vs FP64 CG per system."""
    systems = []
    for g, k in zip(W.batch_grids(), W.BATCH_K_DEFAULT):
        nodes, per = rb.grid_nodes(g, dev)
        rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN, scale=-1.0)
        A64 = rb.Operator(rp, ci, va, nc, dtype="f64", k_max=k)
        A32 = rb.Operator(rp, ci, va, nc, dtype="f32", k_max=k)
        A32_mf = rb.Operator.stencil(nodes, per, scale=-1.0, dtype="f32", k_max=k)
        B = torch.as_tensor(W.zero_mean(W.normal((g.n_cells, k), W.seed_for(4, k, salt=len(systems)))), device=dev)
        systems.append((g, k, A64, A32, B, A32_mf))
    prm = rb.cg_params(rtol=1e-10, mixed=2, project_mean=True, max_sweeps=16)
    batch = rb.Batch([s[2] for s in systems], [s[3] for s in systems], [s[1] for s in systems], prm)
    Bs = [s[4] for s in systems]
    Xs = [torch.zeros_like(b) for b in Bs]
    tuned_ms = batch.tune(Bs, Xs)

    def run_batch():
        for x in Xs:
            x.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = batch.solve(Bs, Xs)
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3, r

    run_batch()
    t_batch, rep = min((run_batch() for _ in range(3)), key=lambda x: x[0])
    # the same batch with the matrix-free inner operators (no matrix streams in the inner solve)
    batch_mf = rb.Batch([s[2] for s in systems], [s[5] for s in systems], [s[1] for s in systems], prm)
    batch_mf.tune(Bs, Xs)

    def run_batch_mf():
        for x in Xs:
            x.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = batch_mf.solve(Bs, Xs)
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3, r

    run_batch_mf()
    t_batch_mf, rep_mf = min((run_batch_mf() for _ in range(3)), key=lambda x: x[0])

    def run_seq(mixed):
        t = 0.0
        its = []
        for g, k, A64, A32, B, _ in systems:
            X = torch.zeros_like(B)
            p = rb.cg_params(rtol=1e-10, mixed=mixed, project_mean=True, check_every=50)
            w = torch.empty(rb.cg_workspace_bytes(A64, k, p), dtype=torch.uint8, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = rb.cg_solve(A64, B, X, A_inner=A32 if mixed else None, params=p, work=w)
            torch.cuda.synchronize()
            t += (time.perf_counter() - t0) * 1e3
            its.append(r.iters)
        return t, its

    run_seq(2)
    t_seq_ir, it_seq = min((run_seq(2) for _ in range(2)), key=lambda x: x[0])
    t_seq_64, it_64 = min((run_seq(0) for _ in range(2)), key=lambda x: x[0])
    return {"systems": [{"grid": g.name, "n": g.n_cells, "k": k} for g, k, *_ in systems],
            "batch_graph_ms": t_batch, "tuned_ms": tuned_ms, "batch_graph_matrix_free_ms": t_batch_mf,
            "batch_matrix_free_true_rel_res": [max(r.true_rel_res) for r in rep_mf],
            "batch_matrix_free_status": [r.status for r in rep_mf], "sequential_ir_ms": t_seq_ir,
            "sequential_fp64_cg_ms": t_seq_64, "speedup_vs_sequential_ir": t_seq_ir / t_batch,
            "speedup_vs_fp64_cg": t_seq_64 / t_batch, "batch_iters": [r.iters for r in rep],
            "batch_true_rel_res": [max(r.true_rel_res) for r in rep], "batch_status": [r.status for r in rep],
            "sequential_ir_iters": it_seq, "fp64_cg_iters": it_64}


def extruded_bench(torch, rb, dev, hbm):
    """Airfoil-shaped mesh (~150k vertices) extruded into 64 periodic planes: the SpMM over the
    k = 64 plane columns vs one SpMV with the same operator assembled as a 3-D CSR."""
    import scipy.sparse as sp

    m = W.airfoil_mesh()
    rp, ci = W.mesh_adjacency(m)
    to = lambda a: torch.as_tensor(a, device=dev)
    vals, area, status = rb.mesh_cot_laplacian(to(m.points), to(m.triangles), to(rp), to(ci))
    nz = W.EXTRUDED_NZ
    dz = W.EXTRUDED_SPAN / nz
    n2 = m.points.shape[0]
    res = {"n2d": n2, "nnz2d": int(ci.shape[0]), "nz": nz, "clamped_edges": int(status[0].item()), "runs": []}
    # the same operator as a 3-D CSR (planes outermost): dz (I (x) L2D) + T_z (x) diag(a / dz)
    L2 = sp.csr_matrix((vals.cpu().numpy(), ci, rp), shape=(n2, n2))
    a = area.cpu().numpy()
    e = np.ones(nz)
    T = sp.diags([e[:-1], -2 * e, e[:-1]], [-1, 0, 1], shape=(nz, nz), format="lil")
    T[0, nz - 1] = 1.0
    T[nz - 1, 0] = 1.0
    L3 = (dz * sp.kron(sp.identity(nz), L2) + sp.kron(T.tocsr(), sp.diags(a / dz))).tocsr()
    L3.sort_indices()
    for dt in ("f64", "f32"):
        tdt = torch.float64 if dt == "f64" else torch.float32
        s = 8 if dt == "f64" else 4
        op = rb.Operator(to(rp), to(ci), vals, n2, dtype=dt, k_max=nz, extruded_nz=nz, z_weight=area / dz, dz=dz)
        X = torch.randn((n2, nz), dtype=tdt, device=dev)
        Y = torch.empty_like(X)
        op.tune(X, Y)
        by = int(ci.shape[0]) * (s + 4) + 4 * (n2 + 1) + s * n2 + 2 * s * n2 * nz
        ms = spmm_ms(torch, op, X, Y, by)
        fl = 2 * int(ci.shape[0]) * nz + 4 * n2 * nz
        op3 = rb.Operator.from_scipy(L3, dtype=dt, k_max=1)
        x1 = torch.randn((L3.shape[0], 1), dtype=tdt, device=dev)
        y1 = torch.empty_like(x1)
        op3.tune(x1, y1)
        by3 = L3.nnz * (s + 4) + 4 * (L3.shape[0] + 1) + 2 * s * L3.shape[0]
        ms3 = spmm_ms(torch, op3, x1, y1, by3)
        res["runs"].append({"dtype": dt, "spmm_k64_ms": ms, "gflops": fl / ms / 1e6, "gbs": by / ms / 1e6,
                            "frac_hbm": by / ms / 1e6 / hbm, "spmv_3d_ms": ms3, "spmv_3d_gbs": by3 / ms3 / 1e6,
                            "speedup_vs_3d_spmv": ms3 / ms, "schedule": op.schedule(X, Y)})
        del op, op3
    return res


def e2e(args, torch, step_items, stream, dev, flops_step):
    """The same step through the public API from pinned host buffers: H2D of every input,
    the six SpMMs, D2H of every result, all inside the timed region.  Uploads, SpMMs and
    downloads run on three streams ordered by events, so that the download of one result
    overlaps the uploads of the next inputs (the host link is full duplex)."""
    hx = [torch.empty(X.shape, dtype=X.dtype, pin_memory=True).copy_(X.cpu()) for (_, _, X, _, _, _) in step_items]
    hy = [torch.empty(Y.shape, dtype=Y.dtype, pin_memory=True) for (_, _, _, Y, _, _) in step_items]
    h2d = sum(t.numel() * t.element_size() for t in hx)
    d2h = sum(t.numel() * t.element_size() for t in hy)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def one():
        done_in, done_op = [], []
        with torch.cuda.stream(s_in):
            for (_, op, X, Y, _, _), a in zip(step_items, hx):
                s_in.wait_stream(stream)  # X's previous readers (last step's SpMM) are done
                X.copy_(a, non_blocking=True)
                done_in.append(torch.cuda.Event())
                done_in[-1].record(s_in)
        for (_, op, X, Y, _, _), ev in zip(step_items, done_in):
            stream.wait_event(ev)
            stream.wait_stream(s_out)  # Y's previous download is done
            op.spmm(X, Y, stream=stream)
            done_op.append(torch.cuda.Event())
            done_op[-1].record(stream)
        with torch.cuda.stream(s_out):
            for (_, op, X, Y, _, _), b, ev in zip(step_items, hy, done_op):
                s_out.wait_event(ev)
                b.copy_(Y, non_blocking=True)
        s_out.synchronize()
        stream.synchronize()

    for _ in range(2):
        one()
    ts = []
    for _ in range(10):
        t = time.perf_counter()
        one()
        ts.append(time.perf_counter() - t)
    ms = statistics.median(ts) * 1e3
    return {"value": flops_step / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "host_link": host_link(torch, dev)}


def host_link(torch, dev, mb=256):
    """The host link's copy rates with pinned buffers of `mb` MB: H2D alone, D2H alone, and both
    at once on two streams (the ceiling of the end-to-end step, whose copies are of this kind)."""
    n = mb * 2 ** 20 // 8
    h_in = torch.empty(n, dtype=torch.float64, pin_memory=True).fill_(1.0)
    h_out = torch.empty(n, dtype=torch.float64, pin_memory=True)
    d_in = torch.empty(n, dtype=torch.float64, device=dev)
    d_out = torch.ones(n, dtype=torch.float64, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
        return statistics.median(ts)

    def both():
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)

    by = n * 8
    t_h2d = timed(lambda: d_in.copy_(h_in, non_blocking=True))
    t_d2h = timed(lambda: h_out.copy_(d_out, non_blocking=True))
    t_both = timed(both)
    return {"bytes": by, "h2d_gbs": by / t_h2d / 1e9, "d2h_gbs": by / t_d2h / 1e9,
            "both_gbs": 2 * by / t_both / 1e9}


def _blocks_for(torch, rb, op, dt, k, dev):
    """Seeded N(0,1) X and an empty Y for op in its type (double-float: split from FP64)."""
    if dt == "df64":
        X = rb.df_split(torch.randn((op.n_cols, k), dtype=torch.float64, device=dev))
        return X, torch.empty((op.n_rows, k, 2), dtype=torch.float32, device=dev)
    tdt = torch.float64 if dt == "f64" else torch.float32
    return (torch.randn((op.n_cols, k), dtype=tdt, device=dev),
            torch.empty((op.n_rows, k), dtype=tdt, device=dev))


def k_sweep(torch, rb, ops, dev, hbm):
    """Laplacian SpMM for k = 1 .. 32 in FP64, FP32 and double-float, CSR and SELL (tuned;
    spmm_ms: graph replays, inputs cycled past the L2).  The double-float column moves FP64's
    bytes (8-byte pairs) and does its arithmetic on the FP32 pipe."""
    res = []
    for dt, fmt in (("f64", "csr"), ("f32", "csr"), ("df64", "csr"), ("f64", "sell"), ("f32", "sell")):
        op, _ = ops[("L" if fmt == "csr" else "L-sell", dt)]
        base = None
        for k in W.ks_sweep():
            X, Y = _blocks_for(torch, rb, op, dt, k, dev)
            op.tune(X, Y)
            s_b = 4 if dt == "f32" else 8
            by = spmm_bytes(op.nnz, op.n_rows, op.n_cols, k, s_b)
            ms = spmm_ms(torch, op, X, Y, by)
            if k == 1:
                base = ms
            res.append({"dtype": dt, "format": fmt, "k": k, "ms": ms, "gflops": 2 * op.nnz * k / ms / 1e6, "gbs": by / ms / 1e6,
                        "frac_hbm": by / ms / 1e6 / hbm, "ai_flop_per_byte": 2 * op.nnz * k / by,
                        "speedup_vs_k_spmv": k * base / ms, "schedule": op.schedule(X, Y)})
            del X, Y
    return res


def step_variants(torch, rb, ops, g, dev, hbm):
    """Two variants of the timed step's kernels, each beside the plain one (spmm_ms: graph
    replays, inputs cycled past the L2): the FP64 SpMMs in double-float arithmetic (the same
    bytes, the multiply-adds on the FP32 pipe), and the gradient with its row-block hint (the
    x-, y- and z-face row blocks taking tiles in turn)."""
    out = {"df64_vs_f64": [], "row_block_hint": []}
    for name in ("L", "G", "M"):
        op64, k = ops[(name, "f64")]
        opdf, _ = ops[(name, "df64")]
        by = spmm_bytes(op64.nnz, op64.n_rows, op64.n_cols, k, 8)
        r = {"op": f"{name}-k{k}"}
        for dt, op in (("f64", op64), ("df64", opdf)):
            X, Y = _blocks_for(torch, rb, op, dt, k, dev)
            op.tune(X, Y)
            ms = spmm_ms(torch, op, X, Y, by)
            r[dt + "_us"] = ms * 1e3
            r[dt + "_frac_hbm"] = by / ms / 1e6 / hbm
            r[dt + "_schedule"] = op.schedule(X, Y)
            del X, Y
        r["speedup"] = r["f64_us"] / r["df64_us"]
        out["df64_vs_f64"].append(r)
    for dt in ("f64", "f32"):
        op, k = ops[("G", dt)]
        X, Y = _blocks_for(torch, rb, op, dt, k, dev)
        by = spmm_bytes(op.nnz, op.n_rows, op.n_cols, k, 8 if dt == "f64" else 4)
        sched = op.schedule(X, Y)
        op.set_schedule(k, sched["vec"], sched["lpr"], 0, -1)  # the direct kernel, with and without the hint
        plain = spmm_ms(torch, op, X, Y, by)
        op.set_row_blocks(face_starts(g))
        hinted = spmm_ms(torch, op, X, Y, by)
        op.set_row_blocks([0])
        op.tune(X, Y)  # back to the tuned schedule for later sections
        out["row_block_hint"].append({"op": f"G-{dt}-k{k}", "plain_us": plain * 1e3, "hint_us": hinted * 1e3})
        del X, Y
    # the three kernel families on every operator of the step, at the tuned vector width with one
    # lane per row: direct (indices and values read by the row's lanes), staged (a block's
    # nonzeros copied to shared memory by its threads first), TMA (a producer warp streaming
    # tiles into a 3-stage shared-memory ring)
    out["schedule_families"] = []
    for name in ("L", "G", "M"):
        for dt in ("f64", "f32"):
            op, k = ops[(name, dt)]
            X, Y = _blocks_for(torch, rb, op, dt, k, dev)
            by = spmm_bytes(op.nnz, op.n_rows, op.n_cols, k, 8 if dt == "f64" else 4)
            op.tune(X, Y)
            tuned = op.schedule(X, Y)
            r = {"op": f"{name}-{dt}-k{k}", "tuned": tuned}
            for fam, stage, gc in (("direct", 0, -1), ("staged", 1, 0), ("tma", 2, 0)):
                op.set_schedule(k, tuned["vec"], 1, stage, gc)
                r[fam + "_us"] = spmm_ms(torch, op, X, Y, by) * 1e3
            op.tune(X, Y)
            out["schedule_families"].append(r)
            del X, Y
    return out


def k_sweep_stencil(torch, rb, g, dev, hbm):
    """The channel Laplacian as a matrix-free operator (rb_fvm_stencil_create: entries formed
    from per-axis tables), k = 1 .. 32, FP32, FP64 and double-float (tuned; spmm_ms: graph
    replays, inputs cycled past the L2):
    algorithmic bytes are X read once and Y written, s k (n_r + n_c), the tables (a few KB)
    aside; beside each, the CSR kernel's time at the same k from `ksweep`."""
    nodes, per = rb.grid_nodes(g, dev)
    res = []
    for dt in ("f32", "f64", "df64"):
        op = rb.Operator.stencil(nodes, per, dtype=dt, k_max=32)
        s_b = 4 if dt == "f32" else 8
        for k in W.ks_sweep():
            X, Y = _blocks_for(torch, rb, op, dt, k, dev)
            op.tune(X, Y)
            by = s_b * k * (op.n_rows + op.n_cols)
            ms = spmm_ms(torch, op, X, Y, by)
            res.append({"dtype": dt, "format": "stencil", "k": k, "ms": ms, "gflops": 2 * op.nnz * k / ms / 1e6,
                        "gbs": by / ms / 1e6, "frac_hbm": by / ms / 1e6 / hbm, "schedule": op.schedule(X, Y)})
            del X, Y
        op.close()
    return res


def time_events(torch, fn, reps):
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(2):
        fn()
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def poisson(torch, rb, ops, g, dev):
    """Poisson solves to a 1e-10 true relative residual on b = M u (k = 3): FP64 CG vs FP32-inner refinement
    (inner operator: the FP32 CSR copy, or the matrix-free Laplacian)."""
    Aop, k = ops[("A", "f64")]
    A32, _ = ops[("A", "f32")]
    Mop, _ = ops[("M", "f64")]
    U = torch.as_tensor(W.face_field(Mop.n_cols, k, 2002), device=dev)
    B = torch.empty((Mop.n_rows, k), dtype=torch.float64, device=dev)
    Mop.spmm(U, B, c=torch.full((k,), -1.0, dtype=torch.float64, device=dev))  # b = -M u
    out = {"k": k, "rtol": 1e-10}
    nodes, per = rb.grid_nodes(g, dev)
    A32_mf = rb.Operator.stencil(nodes, per, scale=-1.0, dtype="f32", k_max=k)  # matrix-free inner operator
    for name, mixed, pers, inner in (("fp64_cg", 0, False, None), ("ir_fp32_inner", 2, False, A32),
                                     ("ir_fp32_inner_persistent", 2, True, A32),
                                     ("ir_fp32_inner_restarted", 1, False, A32),
                                     ("ir_fp32_inner_matrix_free", 2, False, A32_mf)):
        prm = rb.cg_params(rtol=1e-10, mixed=mixed, project_mean=True, check_every=50, persistent=pers)
        work = torch.empty(rb.cg_workspace_bytes(Aop, k, prm), dtype=torch.uint8, device=dev)
        times = []
        for rep in range(2):
            X = torch.zeros((Mop.n_rows, k), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = rb.cg_solve(Aop, B, X, A_inner=inner, params=prm, work=work)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t) * 1e3)
        out[name] = {"ms": min(times), "iters": r.iters, "true_rel_res": r.true_rel_res, "status": r.status,
                     "sweeps": r.sweeps, "spmm_calls": r.spmm_calls, "host_syncs": r.host_syncs}
        if name == "fp64_cg":
            X64 = X.clone()
        else:  # the mixed-precision solution against the FP64 one, per column (both zero-mean)
            out[name]["rel_err_vs_fp64_cg"] = ((X - X64).norm(dim=0) / X64.norm(dim=0)).tolist()
    out["speedup_ir_vs_fp64"] = out["fp64_cg"]["ms"] / out["ir_fp32_inner"]["ms"]
    return out


def multigrid(torch, rb, g, dev, poisson_res=None):
    """Multigrid-preconditioned CG (Sec. 4; Appendix A's level, restriction and prolongation
    SpMMs) to a 1e-10 true relative residual: the channel (k = 3, b = -M u) and the periodic
    128^3 box (k = 8, zero-mean N(0,1)), with the FP64 cycle and with the FP32 cycle inside
    FP64 refinement; beside the Jacobi solvers on the same systems.  Host clock around
    synchronised solves (each solve synchronises to read its report); best of two after one
    untimed solve (which records the CUDA graphs)."""
    out = {"runs": []}
    cases = [("channel-k3", g, 3), ("periodic128-k8", W.unit_periodic_grid(128), 8)]
    for case, grid, k in cases:
        nodes, per = rb.grid_nodes(grid, dev)
        t0 = time.perf_counter()
        m = rb.Multigrid(nodes, per, k_max=k)
        torch.cuda.synchronize()
        t_build = (time.perf_counter() - t0) * 1e3
        if case.startswith("channel"):
            rpm, cim, vam, ncm = rb.fvm_assemble(nodes, per, rb.RB_FVM_DIVERGENCE)
            Mop = rb.Operator(rpm, cim, vam, ncm, dtype="f64", k_max=k)
            U = torch.as_tensor(W.face_field(Mop.n_cols, k, 2002), device=dev)
            B = Mop.spmm(U, c=torch.full((k,), -1.0, dtype=torch.float64, device=dev))
            del Mop, U
        else:
            B = torch.as_tensor(W.zero_mean(W.normal((grid.n_cells, k), W.seed_for(4, k, salt=99))), device=dev)
        for mixed in (False, True):
            prm = rb.mg_params(mixed=mixed)
            X = torch.zeros_like(B)
            m.solve(B, X, prm)
            best = None
            for _ in range(2):
                X.zero_()
                torch.cuda.synchronize()
                t = time.perf_counter()
                r = m.solve(B, X, prm)
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t) * 1e3
                best = (ms, r) if best is None or ms < best[0] else best
            ms, r = best
            out["runs"].append({"case": f"{case}-{'fp32cycle-ir' if mixed else 'fp64'}", "grid": grid.name, "k": k,
                                "levels": m.shapes, "ms": ms, "iters": r.iters, "sweeps": r.sweeps,
                                "true_rel_res": r.true_rel_res, "status": r.status, "build_ms": t_build,
                                "device_gb": m.info().device_bytes / 1e9})
        if case.startswith("periodic"):  # the Jacobi refinement on the same system
            rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN, scale=-1.0)
            A64 = rb.Operator(rp, ci, va, nc, dtype="f64", k_max=k)
            A32 = rb.Operator(rp, ci, va, nc, dtype="f32", k_max=k)
            for name, mixed in (("jacobi-fp64-cg", 0), ("jacobi-ir", 2)):
                p = rb.cg_params(rtol=1e-10, mixed=mixed, project_mean=True, check_every=50)
                w = torch.empty(rb.cg_workspace_bytes(A64, k, p), dtype=torch.uint8, device=dev)
                X = torch.zeros_like(B)
                torch.cuda.synchronize()
                t = time.perf_counter()
                r = rb.cg_solve(A64, B, X, A_inner=A32 if mixed else None, params=p, work=w)
                torch.cuda.synchronize()
                out["runs"].append({"case": f"{case}-{name}", "k": k, "ms": (time.perf_counter() - t) * 1e3,
                                    "iters": r.iters, "true_rel_res": r.true_rel_res})
            del A64, A32
        del m, B
        torch.cuda.empty_cache()
    if poisson_res:
        ch = {r["case"]: r["ms"] for r in out["runs"]}
        out["channel_speedup_vs_jacobi_fp64_cg"] = poisson_res["fp64_cg"]["ms"] / ch["channel-k3-fp32cycle-ir"]
        out["channel_speedup_vs_jacobi_ir"] = poisson_res["ir_fp32_inner"]["ms"] / ch["channel-k3-fp32cycle-ir"]
    return out


def learned_guess(torch, rb, dev, args):
    """Learned initial guess on the Rayleigh-Benard-shaped 128^3 grid (walls in z, tanh 1.4):
    solver-generated pairs (8 forcing sequences solved together, k = 8, by the multigrid CG),
    training with the library's tcgen05 kernels, then CG to 1e-10 on held-out steps from each
    guess (zero, p_{t-1}, the judged network guess, the Galerkin combinations) with the Jacobi
    solvers and the multigrid CG (guess_pipeline.evaluate).  Full configuration by default:
    8 x 252 steps, 1800 training and 200 held-out pairs, 6 epochs."""
    from paper_2508_06710_gb300 import guess_pipeline as gp

    n = W.GUESS_N
    chains = W.GUESS_CHAINS
    full = not args.guess_quick
    steps = W.GUESS_STEPS if full else 40
    holdout = W.GUESS_HOLDOUT if full else 4
    epochs = args.guess_epochs if args.guess_epochs else (6 if full else 3)
    grid = W.rbc_grid(n, 1.4)
    prob = gp.make_problem(torch, grid, chains, dev)
    spectra = W.forcing_spectra(steps, chains, seed=5000)
    Bs, Ps, gen = gp.generate(torch, prob, spectra, W.face_fields, dev)
    train_pairs, _ = gp.pairs(steps, chains, holdout)
    net = gp.network(grid)
    net.init_params(torch.as_tensor(W.normal(net.n_params, 5001).astype(np.float32), device=dev), head_scale=0.1)
    # one forward and one training sample, timed alone
    out1 = torch.empty(prob["n"], dtype=torch.float64, device=dev)
    lacc = torch.zeros(1, dtype=torch.float64, device=dev)
    t_pred = time_events(torch, lambda: net.predict(Bs[3, 0], Ps[2, 0], Ps[1, 0], out=out1), 5)
    t_lg = time_events(torch, lambda: net.loss_grad(Bs[3, 0], Ps[2, 0], Ps[1, 0], Ps[3, 0], loss=lacc), 5)
    net.init_params(torch.as_tensor(W.normal(net.n_params, 5001).astype(np.float32), device=dev), head_scale=0.1)
    tr = gp.train(torch, net, Bs, Ps, train_pairs, epochs=epochs, batch=4, lr=2e-3, lr_final=2e-4, seed=5002)
    ev = gp.evaluate(torch, prob, net, Bs, Ps, range(steps - holdout, steps), chains)
    conv_flops = 0
    for name, kind, ci, co in _unet_layers():
        if kind == "conv3":
            lvl = int(name[3])
            conv_flops += 2 * 27 * ci * co * (prob["n"] >> (3 * lvl))
    return {"grid": f"rbc {n}^3 tanh 1.4", "params": net.n_params, "chains": chains, "steps": steps,
            "holdout": holdout, "full_config": full, "generate": gen,
            "predict_ms": t_pred, "train_sample_ms": t_lg,
            "forward_conv_tflops": conv_flops / (t_pred * 1e-3) / 1e12,
            "train": {k: v for k, v in tr.items()}, "eval": ev}


def _unet_layers(channels=(8, 16, 32, 48)):
    """(name, kind, c_in, c_out) of the guess network (3x3x3 convolutions only matter for the
    flop count)."""
    out = []
    cin = 3
    for l, c in enumerate(channels):
        out += [(f"enc{l}a", "conv3", cin, c), (f"enc{l}b", "conv3", c, c)]
        cin = c
    for l in range(len(channels) - 2, -1, -1):
        out += [(f"up{l}", "up", channels[l + 1], channels[l]), (f"dec{l}a", "conv3", 2 * channels[l], channels[l]),
                (f"dec{l}b", "conv3", channels[l], channels[l])]
    return out


def cpu_baseline(g, budget_s=15.0):
    """The oracle (scipy FP64, one core) on the same step: each SpMM as k separate SpMVs."""
    from oracle import fvm, spmm

    ops = [(fvm.laplacian_direct(g), 3), (fvm.gradient(g), 3), (fvm.divergence(g), 1)]
    Xs = [W.normal((A.shape[1], k), 7 + k) for A, k in ops]
    flops = 0
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s or steps == 0:
        for (A, k), X in zip(ops, Xs):
            spmm.spmm(A, X)
            spmm.spmm(A.astype(np.float32), X.astype(np.float32))
            flops += 2 * 2 * A.nnz * k
        steps += 1
    dt = time.perf_counter() - t0
    out = {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
           "sample": f"{steps} full steps of the same workload (6 SpMMs, scipy CSR, single thread)"}
    # the same oracle on every host core at once: one process per core, each running whole
    # steps for a fixed time (aggregate throughput); spawned, so no process inherits CUDA state
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        rates = pool.map(_oracle_worker, [(g.shape, budget_s / 2)] * cores)
    out["all_cores"] = {"value": sum(rates), "unit": "GFLOP/s", "cores": cores,
                        "sample": f"{cores} processes x {budget_s / 2:.0f} s of whole steps (6 SpMMs each)"}
    return out


def _oracle_worker(arg):
    """One process of the all-core oracle baseline: whole steps for `budget` seconds, GFLOP/s."""
    shape, budget = arg
    import numpy as _np

    from oracle import fvm, spmm

    g = W.channel_grid(*shape, gamma=1.5)
    ops = [(fvm.laplacian_direct(g), 3), (fvm.gradient(g), 3), (fvm.divergence(g), 1)]
    Xs = [W.normal((A.shape[1], k), 7 + k) for A, k in ops]
    flops = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget or flops == 0:
        for (A, k), X in zip(ops, Xs):
            spmm.spmm(A, X)
            spmm.spmm(A.astype(_np.float32), X.astype(_np.float32))
            flops += 2 * 2 * A.nnz * k
    return flops / (time.perf_counter() - t0) / 1e9


def reference_slices(ops, n_slices):
    """Each operator's rows cut into n_slices contiguous CSR slices (the bounded per-step sample)."""
    out = []
    for A, k in ops:
        edges = np.linspace(0, A.shape[0], n_slices + 1).astype(int)
        out.append([(A[edges[i]:edges[i + 1]], k) for i in range(n_slices)])
    return out


def run_reference(args, rank, world, budget_s=120.0):
    """The oracle as it stands (scipy FP64 and FP32 CSR, one core) on the same workload.  A step
    is a bounded sample: 1 / n_slices of every operator's rows (the slices taken in turn, so the
    run covers the whole operators), n_slices chosen from one timed full step so that the whole
    run ends in about `budget_s` seconds; the metric counts the sample's own flops."""
    if rank != 0:
        return None
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    from oracle import fvm, spmm

    ops = [(fvm.laplacian_direct(g), 3), (fvm.gradient(g), 3), (fvm.divergence(g), 1)]
    Xs = [W.normal((A.shape[1], k), 7 + k) for A, k in ops]
    Xs32 = [X.astype(np.float32) for X in Xs]
    t = time.perf_counter()
    for (A, k), X, X32 in zip(ops, Xs, Xs32):
        spmm.spmm(A, X)
        spmm.spmm(A.astype(np.float32), X32)
    t_full = time.perf_counter() - t
    n_slices = max(1, int(np.ceil((args.steps + args.warmup) * t_full / budget_s)))
    sl = reference_slices(ops, n_slices)
    sl32 = [[(A.astype(np.float32), k) for A, k in per] for per in sl]

    def step(i):
        fl = 0
        j = i % n_slices
        for o in range(len(ops)):
            (A, k), (A32, _) = sl[o][j], sl32[o][j]
            spmm.spmm(A, Xs[o])
            spmm.spmm(A32, Xs32[o])
            fl += 2 * 2 * A.nnz * k
        return fl

    for i in range(args.warmup):
        step(i)
    flops = 0
    t = time.perf_counter()
    for i in range(args.steps):
        flops += step(args.warmup + i)
    sec = time.perf_counter() - t
    ms = sec * 1e3 / args.steps
    v = flops / sec / 1e9
    sample = (f"each step 1/{n_slices} of the rows of every operator of the full step (6 SpMMs, scipy CSR, "
              f"single thread), slices in turn")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_cells": g.n_cells, "k": {"L": 3, "G": 3, "M": 1},
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


HEADLINE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                 "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks")


def _pick(d, keys):
    return {k: d[k] for k in keys if d is not None and k in d}


def _round(v, digits=4):
    """Floats of a nested summary to `digits` significant digits (keeps the line short)."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}")
    if isinstance(v, dict):
        return {k: _round(x, digits) for k, x in v.items()}
    if isinstance(v, list):
        return [_round(x, digits) for x in v]
    return v


def headline(out, detail_path):
    """The one short JSON line that ends stdout: the headline metric with its roofline, e2e,
    cpu_baseline and clocks, plus a few figures of the secondary sections; every section in
    full goes to `detail_path`."""
    h = _pick(out, HEADLINE_KEYS)
    if "roofline" in out:
        h["roofline"] = _pick(out["roofline"], ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                                "peak_source", "peak_measured", "frac_of_measured", "hbm_frac_of_measured"))
    if "e2e" in out:
        h["e2e"] = _pick(out["e2e"], ("value", "unit", "ms_per_step", "h2d_bytes_per_step", "d2h_bytes_per_step"))
    if "cpu_baseline" in out:
        cb = out["cpu_baseline"]
        h["cpu_baseline"] = _pick(cb, ("value", "unit", "cores", "kind", "sample"))
        if "all_cores" in cb:
            h["cpu_baseline"]["all_cores"] = _pick(cb["all_cores"], ("value", "cores"))
    s = {}
    if "kernels" in out:
        s["kernel_ms"] = {r["kernel"]: round(r["ms"] * 1e3, 2) for r in out["kernels"]}
        s["kernel_ms_unit"] = "us"
    if "overlapped_step" in out:
        s["overlapped_step_gflops"] = out["overlapped_step"].get("value")
    p = out.get("poisson")
    if p:
        s["poisson_ms"] = {k: v["ms"] for k, v in p.items() if isinstance(v, dict) and "ms" in v}
    mg = out.get("multigrid")
    if mg:
        s["multigrid_ms"] = {r["case"]: r["ms"] for r in mg.get("runs", []) if "case" in r and "ms" in r}
    b = out.get("batch")
    if b:
        s["batch_graph_ms"] = b.get("batch_graph_ms")
        s["batch_graph_matrix_free_ms"] = b.get("batch_graph_matrix_free_ms")
        s["batch_sequential_fp64_cg_ms"] = b.get("sequential_fp64_cg_ms")
    lg = out.get("learned_guess")
    if lg and "eval" in lg:
        s["learned_guess_ms_per_system"] = {k: v.get("ms_per_system") for k, v in lg["eval"].items()
                                            if isinstance(v, dict) and "ms_per_system" in v}
    ks = out.get("ksweep")
    if ks:
        s["ksweep_frac_hbm_csr"] = {f"{r['dtype']}-k{r['k']}": round(r["frac_hbm"], 3) for r in ks if r["format"] == "csr"}
    hl = (out.get("e2e") or {}).get("host_link")
    if hl:
        s["host_link_gbs"] = {"h2d": hl["h2d_gbs"], "d2h": hl["d2h_gbs"], "both": hl["both_gbs"]}
    sv = out.get("step_variants")
    if sv:
        s["df64_vs_f64_us"] = {r["op"]: [r["f64_us"], r["df64_us"]] for r in sv["df64_vs_f64"]}
    kst = out.get("ksweep_stencil")
    if kst:  # the matrix-free sweep at k = 1, 3 and 32
        s["ksweep_stencil_gflops"] = {f"{r['dtype']}-k{r['k']}": round(r["gflops"]) for r in kst if r["k"] in (1, 3, 32)}
    h["summary"] = _round(s)
    h["detail"] = os.path.relpath(detail_path, ROOT) if os.path.isabs(detail_path) else detail_path
    return h


def max_over_ranks(torch, value, world, dev=None):
    """The largest `value` over all ranks (the timing rule of a replicated run)."""
    if world <= 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def profile_run(args):
    """A short, fixed workload for ncu captures (no tuning, no sweeps, no CPU baseline)."""
    import torch

    import paper_2508_06710_gb300 as rb
    from paper_2508_06710_gb300 import build as rbbuild

    rbbuild.build()
    dev = torch.device("cuda", 0)
    if args.profile == "guess":
        # the learned-guess network on the 128^3 Rayleigh-Benard grid: one forward ("predict")
        # and one training pass ("loss_grad") on seeded vectors, each in its NVTX range
        from paper_2508_06710_gb300 import guess_pipeline as gp

        grid = W.rbc_grid(W.GUESS_N, 1.4)
        net = gp.network(grid)
        net.init_params(torch.as_tensor(W.normal(net.n_params, 1).astype(np.float32), device=dev), head_scale=0.1)
        n = net.n
        b, p1, p2, p = (torch.as_tensor(W.normal(n, 10 + i), device=dev) for i in range(4))
        out = torch.empty(n, dtype=torch.float64, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(2):
            net.predict(b, p1, p2, out=out)
            net.loss_grad(b, p1, p2, p, loss=loss)
        torch.cuda.synchronize()
        for name, fn in (("predict", lambda: net.predict(b, p1, p2, out=out)),
                         ("loss_grad", lambda: net.loss_grad(b, p1, p2, p, loss=loss))):
            torch.cuda.nvtx.range_push(name)
            fn()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": args.profile, "ok": True}))
        return
    if args.profile == "mg":
        # one multigrid solve (FP32 cycle inside FP64 refinement) on the channel, k = 3, after
        # an untimed one that records the CUDA graphs; NVTX range "mg_solve"
        g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
        nodes, per = rb.grid_nodes(g, dev)
        m = rb.Multigrid(nodes, per, k_max=3)
        B = torch.as_tensor(W.zero_mean(W.normal((g.n_cells, 3), 2004)), device=dev)
        X = torch.zeros_like(B)
        m.solve(B, X, rb.mg_params(mixed=True))
        X.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("mg_solve")
        r = m.solve(B, X, rb.mg_params(mixed=True))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": args.profile, "ok": True, "iters": r.iters, "res": r.true_rel_res}))
        return
    if args.profile == "stencil":
        # the matrix-free channel Laplacian (rb_fvm_stencil_create), FP32, k = 1 then k = 3,
        # three SpMMs each on seeded blocks
        g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
        nodes, per = rb.grid_nodes(g, dev)
        op = rb.Operator.stencil(nodes, per, dtype="f32", k_max=3)
        for k in (1, 3):
            X = torch.as_tensor(W.normal((g.n_cells, k), 2006).astype(np.float32), device=dev)
            Y = torch.empty_like(X)
            for _ in range(3):
                op.spmm(X, Y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "ok": True}))
        return
    if args.profile == "df":
        # the channel Laplacian in double-float arithmetic, k = 3: three CSR SpMMs, then three
        # matrix-free ones, on seeded blocks
        g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
        nodes, per = rb.grid_nodes(g, dev)
        rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
        X = rb.df_split(torch.as_tensor(W.normal((g.n_cells, 3), 2007), device=dev))
        Y = torch.empty_like(X)
        for op in (rb.Operator(rp, ci, va, nc, dtype="df64", k_max=3), rb.Operator.stencil(nodes, per, dtype="df64", k_max=3)):
            for _ in range(3):
                op.spmm(X, Y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "ok": True}))
        return
    if args.profile == "assembly":
        # the device builds of the 27p Laplacian (96^3 periodic), and of P, R and P^T on the channel
        n = 96
        rb.stencil_assemble((n, n, n), (1.0 / n,) * 3, rb.RB_STENCIL_27P, device=dev)
        rb.stencil_assemble((n, n, n), (1.0 / n,) * 3, rb.RB_STENCIL_13P, device=dev)
        g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
        nodes, per = rb.grid_nodes(g, dev)
        for kind in (rb.RB_REFINE_PROLONG, rb.RB_REFINE_RESTRICT, rb.RB_REFINE_PROLONG_T):
            rb.refine_assemble(nodes, per, kind)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "ok": True}))
        return
    if args.profile == "projection":
        # two Heun RK3 projection steps of m = 2 states on the periodic 128^3 box (multigrid
        # pressure solves); NVTX range "projection_step" around the second
        import math

        from paper_2508_06710_gb300.flow_step import ProjectionStep

        n = 128
        nodes = [torch.linspace(0.0, 2 * math.pi, n + 1, dtype=torch.float64, device=dev) for _ in range(3)]
        st = ProjectionStep(torch, nodes, 2, 0.01, 0.01, mixed=2, solver="mg")
        u = torch.as_tensor(W.normal((n ** 3, 6), 2005), device=dev)
        us = torch.zeros((3 * n ** 3, 2), dtype=torch.float64, device=dev)
        st.step(u, us)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("projection_step")
        st.step(u, us)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": args.profile, "ok": True, "iters": st.iters}))
        return
    if args.profile == "spmm":
        g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
        nodes, per = rb.grid_nodes(g, dev)
        rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
        k, dt = args.profile_k, args.profile_dtype
        op = rb.Operator(rp, ci, va, nc, dtype=dt, k_max=k)
        tdt = torch.float64 if dt == "f64" else torch.float32
        X = torch.ones((op.n_cols, k), dtype=tdt, device=dev)
        Y = torch.empty((op.n_rows, k), dtype=tdt, device=dev)
        if args.profile_sched:
            op.set_schedule(k, *(int(v) for v in args.profile_sched.split(",")))
        for _ in range(3):
            op.spmm(X, Y)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "ok": True, "schedule": op.schedule(X, Y)}))
        return
    g, ops = build_ops(rb, torch, dev)
    if args.profile == "step":
        for name in ("L", "G", "M"):
            for dt in ("f64", "f32"):
                op, k = ops[(name, dt)]
                tdt = torch.float64 if dt == "f64" else torch.float32
                X = torch.ones((op.n_cols, k), dtype=tdt, device=dev)
                Y = torch.empty((op.n_rows, k), dtype=tdt, device=dev)
                for _ in range(args.steps):
                    op.spmm(X, Y)
    else:
        Aop, _ = ops[("A", "f64")]
        A32, _ = ops[("A", "f32")]
        Mop, _ = ops[("M", "f64")]
        nodes, per = rb.grid_nodes(g, dev)
        A32_mf = rb.Operator.stencil(nodes, per, scale=-1.0, dtype="f32", k_max=3)
        for k in (1, 3):
            U = torch.as_tensor(W.face_field(Mop.n_cols, k, 2002), device=dev)
            B = Mop.spmm(U, c=torch.full((k,), -1.0, dtype=torch.float64, device=dev))
            for mixed, inner in ((False, None), (True, A32), (True, A32_mf)):
                prm = rb.cg_params(rtol=1e-10, mixed=mixed, project_mean=True, max_iter=20, check_every=10)
                X = torch.zeros((Mop.n_rows, k), dtype=torch.float64, device=dev)
                rb.cg_solve(Aop, B, X, A_inner=inner, params=prm)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "ok": True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="timed step only (no e2e, sweeps, solves, CPU baseline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-guess", action="store_true", help="skip the learned-guess section")
    ap.add_argument("--guess-quick", action="store_true",
                    help="learned guess on a reduced data set (8 sequences x 40 steps, 3 epochs); the default is "
                         "the full Rayleigh-Benard configuration: 8 sequences x 252 steps (1800 training, 200 test "
                         "pairs), 6 epochs")
    ap.add_argument("--guess-epochs", type=int, default=None)
    ap.add_argument("--nvtx", action="store_true",
                    help="NVTX ranges around the timed region ('timed_step') and each SpMM (its label), for ncu filters")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the dominant kernel, if captured for this build")
    ap.add_argument("--profile", default=None, choices=["step", "cg", "guess", "spmm", "mg", "assembly", "projection", "stencil", "df"],
                    help="short run for an ncu capture: 'step' = the timed step only, 'cg' = a 20-iteration "
                         "FP64 and FP32-refinement Poisson solve (k = 1 and 3), 'guess' = one forward and one "
                         "training pass of the learned-guess network at 128^3 (NVTX 'predict', 'loss_grad'), "
                         "'spmm' = three channel-Laplacian SpMMs with --profile-k columns in --profile-dtype "
                         "on the schedule --profile-sched (vec,lpr,stage,grid_cap; default: the untuned one), "
                         "'mg' = one multigrid solve on the channel (k = 3, NVTX 'mg_solve'), 'assembly' = the 13p / "
                         "27p builds at 96^3 and P, R, P^T on the channel, 'projection' = two projection steps of "
                         "two states at 128^3 (NVTX 'projection_step' around the second), 'stencil' = the "
                         "matrix-free channel Laplacian in FP32, three SpMMs with k = 1 then k = 3, 'df' = the channel "
                         "Laplacian in double-float arithmetic, k = 3, three CSR then three matrix-free SpMMs")
    ap.add_argument("--detail", default=os.path.join(ROOT, "bench_detail.json"),
                    help="file receiving the full result (every section); stdout ends with the headline line only")
    ap.add_argument("--profile-k", type=int, default=32)
    ap.add_argument("--profile-dtype", default="f32", choices=["f64", "f32"])
    ap.add_argument("--profile-sched", default=None)
    args = ap.parse_args()
    if args.profile:
        return profile_run(args)
    rank, world, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3
    if world > 1:
        import torch

        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        if args.impl == "reference":
            print(json.dumps(out))
        else:
            with open(args.detail, "w") as f:
                json.dump(out, f, indent=1)
            print(json.dumps(headline(out, args.detail)))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
