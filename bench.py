#!/usr/bin/env python
"""Throughput of the TR-BRSGD step on one GB300 (and N replicas under torchrun).

Workload (the headline configuration): N=4 tensor 100x100x100x100 FP32
(400 MB), TR ranks all 10, planted cores G_{n(2)} = U_n S V^T with singular
values geometric from 1 to 1e-3, noise of relative norm 1e-4, uniform fiber
sampling, |F| = 1000, fixed step, plain TR-BRSGD.  Inputs are synthetic and
seeded (synth module); X is formed on the device by the library's
reconstruction.  One bench step = one TR-BRSGD iteration (Algorithm 3): mode
draw, Algorithm 2 sampling and fiber gather, residual, gradient (Eq.
S_gradient), update of G_n.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "TR-SGD steps/s & time to rel. error 1e-3 (FP32 vs BF16 vs batched), %roofline"
WORKLOAD_DESC = {
    "c1": "N=3 20^3 FP64, R=3, Gaussian planted cores, noise 1e-3, |F|=50, uniform, fixed step",
    "c2": "N=4 100^4 FP32, R=10, ill-conditioned planted cores, noise 1e-4, |F|=1000, uniform sampling, "
          "plain TR-BRSGD, fixed step",
    "c3": "N=5 40^5 FP32, R=8, Gaussian planted cores, noise 1e-3, |F|=2048, uniform, fixed step",
    "c5": "N=3 1000^3 with X stored in BF16 (2 GB), R=20, ill-conditioned planted cores (1 -> 1e-2), noise 1e-3, "
          "|F|=4096, scaled variant (TR-ScaledBRSGD, h from the same batch) with AdaGrad, BF16 tensor-core "
          "operands, whole-GPU path",
    "c5p": "profiling size of the 1000^3 workload, plain direction: 1000x400x400, R=20, |F|=4096, BF16 operands, "
           "AdaGrad, whole-GPU path",
    "c5ps": "profiling size of c5, scaled variant: 1000x400x400, R=20, |F|=4096, BF16 operands, AdaGrad",
}
DTYPE_NAME = {0: "f64", 1: "f32", 2: "bf16 operands, f32 accumulate"}
UNIT = "steps/s"
L2_BYTES = 129 * 2**20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
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


# ---------------------------------------------------------------------------
# device workload
# ---------------------------------------------------------------------------
def device_problem(w, device, seed_offset=0):
    import torch

    from paper_2303_16492_gb300 import api, synth
    w.seed += seed_offset
    planted = [torch.from_numpy(G).to(device=device, dtype=torch.float32) for G in synth.planted_cores(w)]
    X = api.reconstruct(planted, w.dims, w.ranks)
    gen = torch.Generator(device=device)
    gen.manual_seed(w.seed + 1)
    noise = torch.randn(X.numel(), generator=gen, device=device, dtype=torch.float32)
    xn = torch.linalg.vector_norm(X.double())
    X.add_(noise * (w.noise_rel * xn / torch.linalg.vector_norm(noise.double())).float())
    del noise
    x2 = float(torch.linalg.vector_norm(X.double()) ** 2)
    init = [torch.from_numpy(G).to(device=device, dtype=torch.float32) for G in synth.initial_cores(w, x2)]
    Xtrue = api.reconstruct(planted, w.dims, w.ranks)
    return X, Xtrue, init


# dram__bytes_read.sum + dram__bytes_write.sum per step of a kernel on a
# workload, from one ncu capture (c2: one launch of 200 steps, 99,298,560 B
# read + 1,649,408 B written), with the SHA-256 prefix of the kernel's source
# files at the time of the capture: when the sources differ now, the kernel
# has changed since and the traffic is reported as null
STEP_KERNEL_SOURCES = ["step_kernel.cuh", "blocks.cuh", "common.cuh", "tables.cuh", "df64.cuh", "gramsolve.cuh",
                       "internal.h", "step_f32x3.cu"]
MEASURED_TRAFFIC_PER_STEP = {
    ("c2", "step_cluster_kernel<float,float,12,3,false>"): {"bytes": 504730.88, "sources": "1e8bd39152887ae1"},
}


def sources_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2303_16492_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel):
    rec = MEASURED_TRAFFIC_PER_STEP.get((workload, kernel))
    if rec is None or sources_digest(STEP_KERNEL_SOURCES) != rec["sources"]:
        return None
    return rec["bytes"]


def algorithmic_per_step(w):
    """HBM bytes and flops of one iteration averaged over the modes (uniform
    mode draw): the J sampled fibers (J I_n bytes of X), G_n read and written
    (2 I_n Q, 4 B each) and the other N-1 cores read once (their sampled
    slices come from them); flops 2 J (N-2) R^3 (chain) + 2 I_n Q J (residual)
    + 2 I_n Q J (gradient)."""
    N = len(w.dims)
    sx = 8 if w.prec == 0 else (2 if w.prec == 2 else 4)
    sc = 8 if w.prec == 0 else 4
    by, fl = 0.0, 0.0
    for n in range(N):
        In = w.dims[n]
        Q = w.ranks[n] * w.ranks[(n + 1) % N]
        R = w.ranks[0]
        others = sum(w.dims[k] * w.ranks[k] * w.ranks[(k + 1) % N] for k in range(N) if k != n)
        by += w.J * In * sx + 2 * In * Q * sc + others * sc
        fl += 2 * w.J * (N - 2) * R ** 3 + 4 * In * Q * w.J
    return by / N, fl / N


def method_flops_per_step(w):
    """The residual and gradient contractions of one iteration, 4 I_n Q J flop,
    averaged over the modes."""
    N = len(w.dims)
    return sum(4.0 * w.dims[n] * w.ranks[n] * w.ranks[(n + 1) % N] * w.J for n in range(N)) / N


def measured_fp32_peak():
    """FP32 FMA flop/s of this device, measured now (trsgd_probe_peak)."""
    try:
        from paper_2303_16492_gb300 import api
        return max(api.probe_peak(0, 2048) for _ in range(2))
    except Exception:
        return None


def max_over_ranks(ms, device):
    """The slowest rank's timed milliseconds (all ranks receive it), then a
    barrier; the job's clock is the max over ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(world, steps, ms):
    """Whole-job steps/s: every rank runs `steps` iterations of its own
    problem (replicas, weak scaling) within the max-over-ranks time."""
    return world * steps / (ms * 1e-3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2303_16492_gb300 import api, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    w = synth.workload(args.workload)
    X, Xtrue, init = device_problem(w, device, seed_offset=rank)
    if w.prec == 2:   # BF16-mixed workloads store X in BF16
        X = X.to(torch.bfloat16)
    from paper_2303_16492_gb300 import _abi
    pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=w.prec, alpha=w.alpha, rule=w.rule,
                           eta=w.extra.get("eta_scaled", w.eta) if w.variant else w.eta, variant=w.variant,
                           J_H=w.JH, damping=w.damping, seed=w.seed + 3,
                           x_dtype=_abi.DTYPE_BF16 if w.prec == 2 else None)
    stream = torch.cuda.current_stream()
    solver = api.Solver([pc], [X], [init], stream=stream)
    if args.autotune:
        solver.autotune(steps_per_trial=200)
    cluster, threads = solver.launch_shape()
    solver.run(0, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    l0 = solver.launch_count()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solver.run(args.warmup, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = solver.launch_count() - l0
    clocks = clk.stop()
    if world > 1:
        ms = max_over_ranks(ms, device)
    rse = solver.rel_error(0, Xtrue)
    x_mb = X.numel() * X.element_size() / 1e6
    value = job_throughput(world, args.steps, ms)
    ms_per_step = ms / args.steps

    # roofline of the dominant kernel: the fused step kernel (the only launch in the timed
    # region) on the cluster path; on the whole-GPU path the iteration's contractions
    pk, pk_kind = peaks()
    by, fl = algorithmic_per_step(w)
    if cluster == 0:
        Nw = len(w.dims)
        gemm_fl = method_flops_per_step(w) + (sum(2.0 * (w.JH or w.J) * (w.ranks[n] * w.ranks[(n + 1) % Nw]) ** 2
                                                  for n in range(Nw)) / Nw if w.variant else 0.0)
        achieved = gemm_fl / (ms_per_step * 1e-3) / 1e12
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
        roofline = {"bound": "tensor", "achieved": round(achieved, 3), "peak": peak,
                    "unit": "TFLOP/s", "frac": round(achieved / peak, 5), "traffic": None,
                    "kernel": "whole iteration (samples, tcgen05 contractions, update) over its time",
                    "peak_note": f"dense BF16, {pk_kind} sustained (a kernel sequence inside a long run); "
                                 "flops are the method's 4 I_n Q |F| per iteration"
                                 + ("; FP32 runs them as 6 BF16 piece products" if w.prec == 1 else ""),
                    "algorithmic_flops_per_step": int(gemm_fl)}
    else:
        rmax = next(r for r in (4, 8, 12, 16) if r >= max(w.ranks))
        pieces = solver.tensor_pieces()
        kernel = f"step_cluster_kernel<float,float,{rmax},{pieces},false>"   # plain variant: scaled code compiled out
        # DRAM read+write per step of this kernel on this workload, from one ncu capture
        # (scaled to the timed launch); null when the kernel changed since the capture
        traffic_step = measured_traffic(args.workload, kernel)
        achieved = by / (ms_per_step * 1e-3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        fp32_peak = measured_fp32_peak()
        roofline = {"bound": "hbm", "achieved": round(achieved, 3), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 6),
                    "traffic": None if traffic_step is None else int(traffic_step * args.steps),
                    "traffic_per_step": traffic_step,
                    "kernel": kernel,
                    "peak_note": f"HBM copy bandwidth, {pk_kind}; algorithmic bytes per step = the sampled "
                                 "fibers + G_n read and written + the other N-1 cores read once; one problem "
                                 f"runs on one cluster of {cluster} of the GPU's SMs, latency-bound",
                    "algorithmic_bytes_per_step": int(by), "algorithmic_flops_per_step": int(fl),
                    "fp32_fma": None if fp32_peak is None else {
                        "achieved_tflops": round(fl / (ms_per_step * 1e-3) / 1e12, 4),
                        "peak_tflops_measured": round(fp32_peak / 1e12, 2),
                        "frac": round(fl / (ms_per_step * 1e-3) / fp32_peak, 5)}}

    e2e = run_e2e(args, w, solver, X, init, device) if rank == 0 and not args.no_e2e else None
    ttr = time_to_rse(args, w, device, ms_per_step) if rank == 0 and args.time_to_rse else None
    extras = run_extras(args, device) if rank == 0 and args.extras else None
    cpu = cpu_baseline(args, w) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms_per_step, 6), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME.get(w.prec, "f32"), "data": "synthetic",
               "config": {"workload": f"{args.workload}: {WORKLOAD_DESC.get(args.workload, '')}",
                          "dims": w.dims, "ranks": w.ranks, "J": w.J, "alpha": w.alpha,
                          "parallelism": f"replicas x{world}" if world > 1 else "single problem",
                          "launch": {"cluster_ctas": cluster, "threads": threads, "steps_per_launch": args.steps},
                          "l2": f"inputs larger than L2 (X {x_mb:.0f} MB and its {len(w.dims)} mode-major copies; "
                                "fibers sampled at random each step; the cores stay resident as the iterate)"},
               "rse_after": rse, "roofline": roofline,
               # J * mean_n I_n * bytes(x) per step: the sampled fibers moved per second
               "sampled_fiber_gbs": round(w.J * sum(w.dims) / len(w.dims) * X.element_size() / (ms_per_step * 1e-3) / 1e9,
                                          3),
               "gpu_launches": launches, "clocks": clocks,
               "e2e": e2e, "cpu_baseline": cpu, "time_to_rse": ttr, "extras": extras}
        print(json.dumps(out), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, w, solver_dev, X_dev, init_dev, device):
    """End to end through the public API from host memory: pinned X and
    initial cores on the host, then H2D copies, trsgd_init (mode-major
    copies), K iterations and the D2H read of the cores, all timed."""
    import torch

    from paper_2303_16492_gb300 import api
    Xh = X_dev.cpu().pin_memory()
    ih = [c.cpu().pin_memory() for c in init_dev]
    Xd = torch.empty_like(X_dev)
    cd = [torch.empty_like(c) for c in init_dev]
    outs = [torch.empty(c.shape, dtype=c.dtype, pin_memory=True) for c in init_dev]
    pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=w.prec, alpha=w.alpha, seed=w.seed + 3)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xd.copy_(Xh, non_blocking=True)
    for a, b in zip(cd, ih):
        a.copy_(b, non_blocking=True)
    s = api.Solver([pc], [Xd], [cd], stream=stream)
    s.run(0, args.steps)
    for o, c in zip(outs, cd):
        o.copy_(c, non_blocking=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    h2d = Xh.numel() * Xh.element_size() + sum(c.numel() * c.element_size() for c in ih)
    d2h = sum(c.numel() * c.element_size() for c in outs)
    return {"value": round(args.steps / dt, 2), "unit": UNIT,
            "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": round(d2h / args.steps, 1),
            "note": "X and the initial cores copied from pinned host memory, trsgd_init, K iterations and "
                    "the cores read back, all inside the timed region (bytes amortised per step)"}


def time_to_rse(args, w, device, ms_fp32, target=1e-3, chunk=500, max_steps=60000):
    """Iterations and device seconds until RSE(X_true) <= target (Sec. 4
    stopping rule, checked every `chunk` iterations by trsgd_run; the RSE
    evaluations are not timed), FP32 and BF16-mixed, same inputs and seed."""
    import torch

    from paper_2303_16492_gb300 import api
    out = {"target": target, "check_every": chunk}
    X, Xtrue, init = device_problem(w, device)
    for name, prec in (("fp32", 1), ("bf16_mixed", 2)):
        cores = [c.clone() for c in init]
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=prec, x_dtype=1, alpha=w.alpha, seed=w.seed + 3)
        s = api.Solver([pc], [X], [cores])
        s.run(0, 200)     # warm-up launch (counts toward the iterations)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.run(200, 2000)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 2000
        done, r = s.run(2200, max_steps, chunk=chunk, tol=target, Xref=Xtrue)
        steps = 2200 + done
        out[name] = {"iterations": steps, "reached": bool(0 <= r <= target), "rse": r,
                     "ms_per_iteration": round(ms, 6), "seconds": round(steps * ms * 1e-3, 4)}
        s.close()
    return out


def run_extras(args, device):
    """Secondary measurements (not the headline): other variants of the step."""
    import torch

    from paper_2303_16492_gb300 import api, synth
    out = {}

    def timed(solver, steps):
        solver.run(0, max(50, steps // 10))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        solver.run(10**6, steps)
        b.record()
        torch.cuda.synchronize()
        return steps / (a.elapsed_time(b) * 1e-3)

    try:
        w = synth.workload(args.workload)
        X, Xtrue, init = device_problem(w, device)
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=2, x_dtype=1, alpha=w.alpha, seed=w.seed + 3)
        initb = [c.clone() for c in init]
        s = api.Solver([pc], [X], [initb])
        out["c2_bf16_mixed_tensor_core_steps_per_s"] = round(timed(s, 20000), 1)
        out["c2_bf16_mixed_rse_after"] = s.rel_error(0, Xtrue)
        s.close()
        # FP32 contractions on the FMA units instead of three BF16 pieces on the tensor cores
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, seed=w.seed + 3,
                               fp32_units=api._abi.FP32_FMA)
        initf = [c.clone() for c in init]
        s = api.Solver([pc], [X], [initf])
        out["c2_fp32_fma_units_steps_per_s"] = round(timed(s, 20000), 1)
        out["c2_fp32_fma_units_rse_after"] = s.rel_error(0, Xtrue)
        s.close()
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=0.5, variant=1, damping=1e-9,
                               seed=w.seed + 3)
        s = api.Solver([pc], [X], [init])
        out["c2_scaled_fp32_steps_per_s"] = round(timed(s, 2000), 1)
        s.close()
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, dist=2, seed=w.seed + 3)
        init2 = [c.clone() for c in init]
        s = api.Solver([pc], [X], [init2])
        out["c2_euclidean_fp32_steps_per_s"] = round(timed(s, 5000), 1)
        s.close()
        del X, Xtrue
    except Exception as e:  # extras never hide the headline
        out["error"] = repr(e)
    try:
        out.update(run_batched(args, device))
    except Exception as e:
        out["batched_error"] = repr(e)
    try:
        out.update(run_c3(args, device))
    except Exception as e:
        out["c3_error"] = repr(e)
    try:
        out.update(run_large(args, device))
    except Exception as e:
        out["c5_error"] = repr(e)
    try:
        out["paper_experiment_shapes"] = run_paper_shapes(args, device)
    except Exception as e:
        out["paper_shapes_error"] = repr(e)
    try:
        out["experiment_2"] = run_exp2(args, device)
    except Exception as e:
        out["experiment_2_error"] = repr(e)
    try:
        out["full_gradient_e1"] = run_full_gradient(args, device)
    except Exception as e:
        out["full_gradient_error"] = repr(e)
    return out


def run_full_gradient(args, device, iters=50):
    """The full-gradient methods the paper compares against, on Experiment I
    (300^3, R = 10) with the paper's steps (TR-GD alpha = 6e-7, TR-ScaledGD
    alpha = 0.5): iterations/s (device events over `iters` iterations, each
    updating all three cores from the same iterate) and the RSE reached, next
    to TR-BRSGD's steps/s on the same problem (the per-iteration contrast of
    Sec. 4)."""
    import torch

    from paper_2303_16492_gb300 import api, synth
    w = synth.workload("e1")
    X, Xtrue, init = device_problem(w, device)
    out = {"iterations": iters}
    for label, scaled, alpha in (("TR-GD", False, 6e-7), ("TR-ScaledGD", True, 0.5)):
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, seed=w.seed + 3)
        s = api.Solver([pc], [X], [[c.clone() for c in init]])
        try:
            s.gd_step(scaled=scaled, alpha=alpha)   # scratch allocation and warm-up
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(iters):
                s.gd_step(scaled=scaled, alpha=alpha)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            out[label] = {"alpha": alpha, "iterations_per_s": round(iters / (ms * 1e-3), 1),
                          "ms_per_iteration": round(ms / iters, 4), "rse_after": s.rel_error(0, Xtrue)}
        except Exception as e:
            out[label] = {"error": repr(e)}
        s.close()
    del X, Xtrue, init
    return out


def run_exp2(args, device):
    """Experiment II of Sec. 4 at 300^3 (dims unstated in the paper): for each
    condition number kappa in {1e2, 1e4, 1e6}, TR-BRSGD (alpha 5e-4) and
    TR-ScaledBRSGD (alpha 9e-2, |H| = 1200), each with the uniform, Euclidean
    and leverage distributions, |F| = 200, R = 5, run for a wall-clock budget
    (the paper's MT = 10 s; `--exp2-seconds`) from the same initial cores:
    iterations done and the RSE reached (or the error a diverging run raised)."""
    import torch

    from paper_2303_16492_gb300 import api, synth
    out = {"seconds_per_run": args.exp2_seconds}
    for base in synth.EXP2_WORKLOADS:
        w = synth.workload(base)
        X, Xtrue, init = device_problem(w, device)
        res = {}
        for variant_name in (base, base + "-s"):
            wv = synth.workload(variant_name)
            for dist_name, dist in (("U", 0), ("E", 2), ("L", 1)):
                label = ("TR-ScaledBRSGD-" if wv.variant else "TR-BRSGD-") + dist_name
                pc = api.ProblemConfig(dims=wv.dims, ranks=wv.ranks, J=wv.J, prec=1, alpha=wv.alpha,
                                       variant=wv.variant, J_H=wv.JH, dist=dist, seed=wv.seed + 3)
                s = api.Solver([pc], [X], [[c.clone() for c in init]])
                try:
                    t0 = time.perf_counter()
                    done, _ = s.run(0, 10**9, chunk=250, max_seconds=args.exp2_seconds)
                    torch.cuda.synchronize()
                    sec = time.perf_counter() - t0
                    res[label] = {"iterations": int(done), "seconds": round(sec, 3),
                                  "rse": s.rel_error(0, Xtrue)}
                except Exception as e:
                    res[label] = {"error": repr(e)}
                s.close()
        out[f"kappa={1.0 / w.smin:.0e}"] = res
        del X, Xtrue, init
    return out


def run_paper_shapes(args, device):
    """The shapes of the paper's experiments (Sec. 4): Experiment I (300^3,
    R=10, |F|=200, plain and scaled with |H| = 200 / 400) run for the paper's
    T = 4000 iterations, and same-shape stand-ins for the three hyperspectral
    images (plain and scaled with |H| = 1000) for 2000 iterations.  Steps/s of
    the timed run (device events) and the RSE it reached."""
    import torch

    from paper_2303_16492_gb300 import api, synth
    out = {}
    for name in synth.NEXT_WORKLOADS:
        w = synth.workload(name)
        X, Xtrue, init = device_problem(w, device)
        steps = 4000 if name.startswith("e1") else 2000
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, variant=w.variant,
                               J_H=w.JH, damping=w.damping, seed=w.seed + 3)
        rec = {"dims": w.dims, "R": w.ranks[0], "J": w.J, "J_H": w.JH, "variant": "scaled" if w.variant else "plain",
               "alpha": w.alpha, "iterations": steps}
        s = api.Solver([pc], [X], [[c.clone() for c in init]])
        try:
            rec["rse_start"] = round(s.rel_error(0, Xtrue), 6)
            shape = s.launch_shape()
            rec["launch"] = {"cluster_ctas": shape[0], "threads": shape[1], "tensor_pieces": s.tensor_pieces()}
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s.run(0, steps)
            b.record()
            torch.cuda.synchronize()
            rec["steps_per_s"] = round(steps / (a.elapsed_time(b) * 1e-3), 1)
            rec["rse_after"] = s.rel_error(0, Xtrue)
        except Exception as e:   # a diverging step size is reported, not hidden
            rec["error"] = repr(e)
        s.close()
        out[name] = rec
        del X, Xtrue, init
    return out


def run_c3(args, device):
    """The c3 workload (N=5, 40^5, R=8, |F|=2048) with each of the four
    distributions (steps/s and RSE after the timed iterations), and the
    sampled-loss adjoint of all five cores (launches/s)."""
    import torch

    from paper_2303_16492_gb300 import api, synth
    w = synth.workload("c3")
    X, Xtrue, init = device_problem(w, device)
    out = {}
    for name, dist, steps in (("uniform", 0, 3000), ("leverage", 1, 1000), ("euclidean", 2, 1000),
                              ("optimal", 3, 40)):
        cores = [c.clone() for c in init]
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, dist=dist, seed=w.seed + 3)
        s = api.Solver([pc], [X], [cores])
        s.run(0, max(10, steps // 10))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.run(10**5, steps)
        b.record()
        torch.cuda.synchronize()
        out[f"c3_{name}_steps_per_s"] = round(steps / (a.elapsed_time(b) * 1e-3), 1)
        s.close()
    # adjoint of the sampled loss for all cores at |F| = 2048
    n = 2
    idx = torch.randint(0, w.dims[0], (w.J, 5), device=device, dtype=torch.int32)
    XS = torch.randn(w.J, w.dims[n], device=device)
    wt = torch.ones(w.J, device=device)
    api.sampled_loss_grad(init, w.dims, w.ranks, n, idx, XS, wt)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(200):
        api.sampled_loss_grad(init, w.dims, w.ranks, n, idx, XS, wt)
    b.record()
    torch.cuda.synchronize()
    out["c3_adjoint_all_cores_per_s"] = round(200 / (a.elapsed_time(b) * 1e-3), 1)
    del X, Xtrue
    return out


def run_large(args, device, target=1e-2, check=100, max_steps=4000, timed_steps=500):
    """The large workload (N=3, 1000^3, R=20, |F|=4096, AdaGrad) on the
    whole-GPU path as its recipe states it: the scaled variant (Sec. 3.3) with
    the adaptive step, BF16 tensor-core contractions with X stored in BF16
    (2 GB) against the FP32 path (X in FP32, three BF16 pieces per operand);
    the plain direction beside it.  Steps/s and iterations / device seconds
    until RSE (against the noiseless tensor) <= target, checked every `check`
    iterations (evaluations not timed).  Tensor rate: the method's flops,
    4 I_n Q |F| per iteration (plus 2 |H| Q^2 for the scaled variant's Gram),
    over the iteration time, against the measured sustained BF16 peak."""
    import torch

    from paper_2303_16492_gb300 import _abi, api, synth
    w = synth.workload("c5")
    X, Xtrue, init = device_problem(w, device)
    Xb = X.to(torch.bfloat16)
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
    out = {}
    N = len(w.dims)
    gemm_flops = method_flops_per_step(w)
    gram_flops = sum(2.0 * w.J * (w.ranks[n] * w.ranks[(n + 1) % N]) ** 2 for n in range(N)) / N
    for label, prec, variant in (("bf16_scaled", _abi.BF16_MIXED, 1), ("fp32_scaled", _abi.FP32, 1),
                                 ("bf16_plain", _abi.BF16_MIXED, 0), ("fp32_plain", _abi.FP32, 0)):
        bf = prec == _abi.BF16_MIXED
        cores = [c.clone() for c in init]
        pc = api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=prec,
                               x_dtype=_abi.DTYPE_BF16 if bf else _abi.DTYPE_F32, rule=w.rule,
                               eta=w.extra.get("eta_scaled", w.eta) if variant else w.eta, variant=variant,
                               seed=w.seed + 3)
        s = api.Solver([pc], [Xb if bf else X], [cores])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ms_total, it, rse, reached = 0.0, 0, None, False
        try:
            while it < max_steps:
                a.record()
                s.run(it, check)
                b.record()
                torch.cuda.synchronize()
                ms_total += a.elapsed_time(b)
                it += check
                rse = s.rel_error(0, Xtrue)
                if rse <= target:
                    reached = True
                    break
            a.record()
            s.run(it, timed_steps)
            b.record()
            torch.cuda.synchronize()
        except Exception as ex:   # a numerical failure of the run is reported, not hidden
            out[f"c5_{label}"] = {"error": str(ex), "iterations": it}
            s.close()
            continue
        ms = a.elapsed_time(b) / timed_steps
        s.close()
        fl = gemm_flops + (gram_flops if variant else 0.0)
        out[f"c5_{label}"] = {
            "steps_per_s": round(1e3 / ms, 1), "us_per_step": round(ms * 1e3, 2),
            "time_to_rse": {"target": target, "iterations": it, "reached": reached, "rse": rse,
                            "seconds": round(ms_total * 1e-3, 4)},
            "method_tflops": round(fl / (ms * 1e-3) / 1e12, 2),
            "frac_of_bf16_sustained": round(fl / (ms * 1e-3) / 1e12 / peak, 4),
            "sampled_fiber_gbs": round(w.J * sum(w.dims) / len(w.dims) * (2 if bf else 4) / (ms * 1e-3) / 1e9, 2)}
    out["c5_config"] = {"dims": w.dims, "ranks": w.ranks, "J": w.J, "rule": "AdaGrad", "eta_plain": w.eta,
                        "eta_scaled": w.extra.get("eta_scaled", w.eta), "path": "grid (whole GPU)",
                        "x_storage": "BF16 (2 GB) for the BF16 runs; FP32 (4 GB) for the FP32 runs",
                        "peak": f"{peak} TFLOP/s dense BF16, {pk_kind} sustained"}
    del X, Xb, Xtrue
    return out


def batched_problems(device, count=64):
    """Batched recipe: 64 independent N=3 problems, I_n ~ U{30..200},
    R_n ~ U{4..16}, Gaussian planted cores, noise 1e-3, |F| = 256 each."""
    import torch

    from paper_2303_16492_gb300 import api, synth
    ws = synth.batched_workloads(count)
    Xs, inits, pcs, Xts = [], [], [], []
    for w in ws:
        planted = [torch.from_numpy(G).to(device=device, dtype=torch.float32) for G in synth.planted_cores(w)]
        Xt = api.reconstruct(planted, w.dims, w.ranks)
        gen = torch.Generator(device=device)
        gen.manual_seed(w.seed + 1)
        nz = torch.randn(Xt.numel(), generator=gen, device=device, dtype=torch.float32)
        X = Xt + nz * (w.noise_rel * torch.linalg.vector_norm(Xt) / torch.linalg.vector_norm(nz))
        x2 = float(torch.linalg.vector_norm(X.double()) ** 2)
        inits.append([torch.from_numpy(G).to(device=device, dtype=torch.float32) for G in synth.initial_cores(w, x2)])
        Xs.append(X)
        Xts.append(Xt)
        pcs.append(api.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, seed=w.seed + 3))
    return ws, pcs, Xs, Xts, inits


def run_batched(args, device, steps=2000):
    import torch

    from paper_2303_16492_gb300 import api
    ws, pcs, Xs, Xts, inits = batched_problems(device)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    s = api.Solver(pcs, Xs, inits, stream=side)
    s.autotune(steps_per_trial=50)   # cluster size and threads per problem cluster
    shape = s.launch_shape()
    # one persistent launch of `chunk` iterations of all 64 problems, captured in a CUDA
    # graph; the device-resident iteration counter advances on every replay
    chunk = 250
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        s.step_counter(chunk)
    s.set_counter(0)
    with torch.cuda.stream(side):   # replays go to the current stream: keep them on the handle's
        for _ in range(2):
            g.replay()
    torch.cuda.synchronize()
    reps = max(1, steps // chunk)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(side):
        a.record(side)
        for _ in range(reps):
            g.replay()
        b.record(side)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) * 1e-3
    steps = reps * chunk
    rse = [s.rel_error(p, Xts[p]) for p in range(0, len(ws), 16)]
    s.close()
    # HBM bytes of one round (every problem one iteration), as for one problem
    round_bytes = sum(algorithmic_per_step(w)[0] for w in ws)
    pk, pk_kind = peaks()
    gbs = round_bytes * steps / sec / 1e9
    # time to RSE 1e-3 (against each problem's noiseless tensor) of the batched form: fresh
    # cores, graph replays of 250 iterations until every problem is there (evaluations untimed)
    cores = [[c.clone() for c in cs] for cs in inits]
    s = api.Solver(pcs, Xs, cores, stream=side)
    s.autotune(steps_per_trial=50)   # the same choice (trial steps leave the cores unchanged)
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=side):
        s.step_counter(chunk)
    s.set_counter(0)
    torch.cuda.synchronize()
    done, ms_total, it, todo = [False] * len(ws), 0.0, 0, set(range(len(ws)))
    first = [None] * len(ws)
    while todo and it < 40 * chunk:
        with torch.cuda.stream(side):
            a.record(side)
            g2.replay()
            b.record(side)
        torch.cuda.synchronize()
        ms_total += a.elapsed_time(b)
        it += chunk
        for p in sorted(todo):
            if s.rel_error(p, Xts[p]) <= 1e-3:
                first[p] = it
                todo.discard(p)
    s.close()
    return {"c4_batched_problem_steps_per_s": round(len(ws) * steps / sec, 1),
            "c4_batched_rounds_per_s": round(steps / sec, 1), "c4_launch_shape": list(shape),
            "c4_execution": "autotuned shape; the problems' clusters in order of decreasing work; one persistent "
                            "launch of 250 iterations of all problems per CUDA-graph replay",
            "c4_rse_sample": [float(f"{r:.3e}") for r in rse],
            "c4_roofline": {"bound": "hbm", "achieved": round(gbs, 2), "peak": pk.get("hbm_gbs", 6800.0),
                            "unit": "GB/s", "frac": round(gbs / pk.get("hbm_gbs", 6800.0), 5),
                            "algorithmic_bytes_per_round": int(round_bytes),
                            "note": f"fibers + G_n read and written + the other cores, every problem; {pk_kind} peak"},
            "c4_time_to_rse_1e-3": {"all_reached": not todo, "iterations_all": it if not todo else None,
                                    "device_seconds": round(ms_total * 1e-3, 4),
                                    "reached": len(ws) - len(todo), "problems": len(ws),
                                    "median_iterations": sorted(x for x in first if x is not None)[
                                        (len(ws) - len(todo)) // 2] if len(ws) > len(todo) else None}}


def cpu_baseline(args, w, budget_s=None):
    """The FP64 oracle, as it stands, timed on the host cores over a bounded
    sample of iterations of the same workload."""
    from oracle import brsgd as ob
    from oracle import tr
    from paper_2303_16492_gb300 import synth
    budget_s = budget_s or args.cpu_seconds
    planted = synth.planted_cores(w)
    N = len(w.dims)
    P = [tr.fold2(G, w.ranks[n], w.ranks[(n + 1) % N]) for n, G in enumerate(planted)]
    Xt = tr.reconstruct(P)
    noise = synth.noise(w.dims, w.seed + 1).reshape(w.dims, order="F")
    X = Xt + noise * (w.noise_rel * np.linalg.norm(Xt) / np.linalg.norm(noise))
    del noise, Xt
    init = synth.initial_cores(w, float(np.sum(X * X)))
    st = ob.State.new([tr.fold2(G, w.ranks[n], w.ranks[(n + 1) % N]) for n, G in enumerate(init)])
    cfg = ob.Config(J=w.J, alpha=w.alpha, seed=w.seed + 3)
    ob.step(st, X, cfg, 0)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < budget_s:
        ob.step(st, X, cfg, 1 + n)
        n += 1
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": round(n / dt, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle iterations of the same workload in {dt:.1f} s (python FP64, numpy BLAS "
                      f"threads up to {cores})"}


def run_reference(args):
    """--impl reference: the oracle timed as the reference arm (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2303_16492_gb300 import synth
    w = synth.workload(args.workload)
    per_step_budget = max(5.0, args.cpu_seconds)
    cpu = cpu_baseline(args, w, budget_s=per_step_budget)
    value = cpu["value"]
    steps = int(min(args.steps, max(1, value * per_step_budget)))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": steps, "warmup": 1,
           "ms_per_step": round(1e3 / value, 3) if value else None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{args.workload} (same synthetic workload as the GPU arm)"},
           "cpu_baseline": cpu,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--warmup", type=int, default=2000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--time-to-rse", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--exp2-seconds", type=float, default=0.25,
                    help="wall-clock budget per run of the Experiment II sweep in the extras (the paper: 10)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
