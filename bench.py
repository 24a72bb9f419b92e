#!/usr/bin/env python
"""Benchmark: MCMC samples/s to the converged fixed point on GB300, against a sequential GPU
loop, for MALA on Bayesian logistic regression (N=1000 rows, D=25, T=16384, FP32, tol 1e-5).

One "step" is one full parallel-Newton solve of the chain (all Newton iterations: evaluate and
linearise, scan, residual check) on inputs already resident in HBM.  The L2 cache is flushed
(a 512 MB write) before every timed step, outside the timed interval.  Under torchrun each rank
solves its own chain (independent noise) on its own GPU: weak scaling, no collective on the
data path; the reported time is the max over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "MCMC samples/s to converged fixed point (tol stated) on 1 GB300 vs sequential GPU loop"
UNIT = "samples/s"
WL = W.C2
CLIP = 1            # clip J to [-1, 1] (Appendix B.4): the step 0.01 makes I + eps H expanding
JAC = "diag"        # quasi-DEER with the exact diagonal (of the held-gate Jacobian by default)
WORKLOAD = (f"{WL.name}: MALA on synthetic logistic regression (N={WL.N}, D={WL.D}), "
            f"T={WL.T}, step {WL.step}, FP32, quasi-DEER exact diagonal, clip, tol {WL.tol}")

# FP32 FMA peak of the GB300 (no tensor cores): 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic flops of one evaluate-and-linearise launch (MALA, exact diagonal), per timestep:
# 2 gradients (2 N D MACs each) and diag(X^T W X) (N D MACs) = 5 N D MACs = 10 N D flops; with
# the stop-gradient gate term add two Hessian-vector products (2 N D MACs each): 18 N D flops.
def alg_flops_per_t(gate_grad: int) -> int:
    return (18 if gate_grad else 10) * WL.N * WL.D


def tensor_peak_fp32_equiv():
    """The tensor-core kernel computes its FP32 contractions as three tf32 products; its peak in
    FP32-equivalent flops is the tf32 dense rate / 3, the tf32 rate being the measured bf16 rate
    x the nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        bf16 = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
        src = "measured bf16 (MEASURED_PEAKS.json)"
    except Exception:
        bf16, src = 1900.0, "fallback bf16 1.9 PFLOP/s"
    return bf16 * (1.1 / 2.25) / 3.0, src


# DRAM traffic of one launch of the dominant kernel (eval_logreg_tc_kernel) from the committed
# ncu capture (profiles/eval_logreg_tc_c2.md): 4.16 MB read, 0 written (the outputs stay in L2).
EVAL_TRAFFIC_BYTES = 4159744


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-variants", action="store_true", help="skip the dense-Newton line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c1", "c3_diag", "c3_bf16", "c3_block", "c4", "c5",
                             "gibbs_diag", "gibbs_dense", "adjoint_small", "c3_paper",
                             "scan_sweep"],
                    help="c2 (default) is the headline line; the others measure the other "
                         "configurations")
    ap.add_argument("--basis", action="store_true",
                    help="solve in the eigenbasis of X^T X (Section 3.4 reparameterisation)")
    ap.add_argument("--gate-grad", type=int, default=0,
                    help="1: the stop-gradient gate term of Section 3.2 in J")
    ap.add_argument("--scan-log2", default="20,22,24,26,28",
                    help="scan_sweep: log2 of the element counts T*D")
    ap.add_argument("--scan-d", type=int, default=8, help="scan_sweep: channels D")
    ap.add_argument("--scan-t", default=None,
                    help="scan_sweep: comma list of T (overrides --scan-log2)")
    ap.add_argument("--scan-precisions", default="f32,f32_scan_bf16",
                    help="scan_sweep: precisions")
    ap.add_argument("--c5-seq-after", type=int, default=150,
                    help="c5: Newton sweeps after which an unconverged chain is completed by the "
                         "sequential loop (0: Newton only)")
    ap.add_argument("--scan-kernel", choices=["rows", "staged", "pipe", "pipe2"], default=None,
                    help="diagonal scan kernel for D <= 32 (default: the library's choice)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(dist, world, device, ms, launches, e2e_ms):
    """Whole-job figures from per-rank ones: the step time and the end-to-end time are the max
    over ranks (the job ends with its slowest rank), launches are summed.  Every rank gets the
    same answer; with one rank the inputs come back unchanged."""
    import torch
    if world <= 1:
        return float(ms), int(launches), float(e2e_ms)
    t = torch.tensor([ms, e2e_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(launches)], device=device, dtype=torch.float64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t[0].item()), int(n.item()), float(t[1].item())


def job_value(world, T, ms):
    """samples/s of the whole job: every rank solves its own chain of T steps (weak scaling)."""
    return world * T / (ms / 1000.0)


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle's sequential chain on the host cores (bounded sample)
# ------------------------------------------------------------------------------------------
def oracle_rate(min_seconds: float, max_steps: int | None = None):
    import oracle as O
    X, y, _ = W.blr_data(WL.N, WL.D, seed=WL.seed)
    xi, u = W.noise(WL.T, WL.D, seed=0, dtype=np.float32)
    steps = WL.T if max_steps is None else min(WL.T, max_steps)
    p = O.Problem(O.Target("logreg", WL.D, X=X, y=y, sigma_p=1.0), "mala", WL.step,
                  xi=xi[:steps].astype(np.float64), u=u[:steps])
    done, t0 = 0, time.perf_counter()
    while True:
        O.chain(p, steps, np.zeros(WL.D))
        done += steps
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return done / el, done, el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each bench step: one bounded sample (2048 steps of the chain) of the oracle
    for _ in range(args.warmup):
        oracle_rate(0.0, max_steps=2048)
    times = []
    samples = 0
    for _ in range(args.steps):
        r, n, el = oracle_rate(0.0, max_steps=2048)
        times.append(el)
        samples += n
    total = sum(times)
    value = samples / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "first 2048 steps of the chain per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "first 2048 steps of the same chain, per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2508_18413_gb300 as P

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    X, y, _ = W.blr_data(WL.N, WL.D, seed=WL.seed, dtype=np.float32)
    xi_h, u_h = W.noise(WL.T, WL.D, seed=rank, dtype=np.float32)   # one chain per rank
    Xd = torch.tensor(X, device=dev)
    yd = torch.tensor(y, device=dev)
    xid = torch.tensor(xi_h, device=dev)
    ud = torch.tensor(u_h, device=dev)
    s0 = torch.zeros(WL.D, dtype=torch.float32, device=dev)
    Qd = None
    if args.basis:
        _, Qh = np.linalg.eigh(X.astype(np.float64).T @ X.astype(np.float64))
        Qd = torch.tensor(Qh.astype(np.float32), device=dev)
    tgt = P.Target("logreg", WL.D, X=Xd, y=yd, prior_scale=1.0, Q=Qd)
    opt = P.Options(sampler="mala", step=WL.step, jac=JAC, precision="f32", atol=WL.tol,
                    clip=CLIP, gate_grad=args.gate_grad)
    s_out = torch.empty((WL.T, WL.D), dtype=torch.float32, device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)  # 512 MB > L2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        _, res = P.pmcmc_solve(tgt, opt, WL.T, s0, xi=xid, u=ud, s_out=s_out)
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    step_ms, results = [], []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, res = P.pmcmc_solve(tgt, opt, WL.T, s0, xi=xid, u=ud, s_out=s_out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        results.append(res)
    barrier()
    clk = clocks.stop()
    # kernel durations: the same solves with per-launch CUDA events (host-driven loop)
    P.pmcmc_profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        P.pmcmc_solve(tgt, opt, WL.T, s0, xi=xid, u=ud, s_out=s_out)
    torch.cuda.synchronize()
    prof = P.pmcmc_profile_get()
    P.pmcmc_profile_enable(False)
    # launches inside the timed region: one evaluate per iteration plus one per solve, one
    # scan per iteration, one control kernel per evaluate, and the solve's set-up kernels
    launches_timed = sum(3 * r["iters"] + 2 + 5 for r in results)

    ms_local = sum(step_ms) / len(step_ms)

    # --- end to end through the public API with host buffers (pinned) ---------------------
    Xh = torch.tensor(X).pin_memory()
    yh = torch.tensor(y).pin_memory()
    xih = torch.tensor(xi_h).pin_memory()
    uh = torch.tensor(u_h).pin_memory()
    s0h = torch.zeros(WL.D, dtype=torch.float32).pin_memory()
    outh = torch.empty((WL.T, WL.D), dtype=torch.float32).pin_memory()
    Xe, ye, xie, ue, s0e = (torch.empty_like(t, device=dev) for t in (Xh, yh, xih, uh, s0h))
    tgt_e = P.Target("logreg", WL.D, X=Xe, y=ye, prior_scale=1.0, Q=Qd)
    h2d = sum(t.numel() * t.element_size() for t in (Xh, yh, xih, uh, s0h))
    d2h = outh.numel() * outh.element_size()
    e2e_ms = []
    barrier()
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d_, h_ in ((Xe, Xh), (ye, yh), (xie, xih), (ue, uh), (s0e, s0h)):
            d_.copy_(h_, non_blocking=True)
        so, _ = P.pmcmc_solve(tgt_e, opt, WL.T, s0e, xi=xie, u=ue, s_out=s_out)
        outh.copy_(so, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    barrier()
    ms, launches, e2e = combine_ranks(dist, world, dev, ms_local, launches_timed,
                                      statistics.mean(e2e_ms))
    value = job_value(world, WL.T, ms)

    # --- sequential GPU loop (the speedup denominator) --------------------------------------
    seq_ms = None
    if rank == 0:
        P.pmcmc_seq_solve(tgt, opt, WL.T, s0, xid, ud)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        P.pmcmc_seq_solve(tgt, opt, WL.T, s0, xid, ud)
        e1.record(stream)
        e1.synchronize()
        seq_ms = e0.elapsed_time(e1)

    # --- dense-Newton line (same chain) ------------------------------------------------------
    dense = None
    if rank == 0 and not args.no_variants:
        optd = P.Options(sampler="mala", step=WL.step, jac="dense", precision="f32", atol=WL.tol,
                         clip=CLIP, max_iters=300)
        P.pmcmc_solve(tgt, optd, WL.T, s0, xi=xid, u=ud, s_out=s_out)
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, rd = P.pmcmc_solve(tgt, optd, WL.T, s0, xi=xid, u=ud, s_out=s_out)
        e1.record(stream)
        e1.synchronize()
        dms = e0.elapsed_time(e1)
        dense = {"value": WL.T / (dms / 1000.0), "unit": UNIT, "ms": dms, "newton_iters": rd["iters"],
                 "status": rd["status"]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu:
        rate, nsamp, el = oracle_rate(10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nsamp} steps (whole chain repeated) of the same workload in FP64, "
                         f"{el:.1f} s"}

    avg_eval_ms = prof["eval_ms"] / max(1, prof["eval_launches"])
    achieved = alg_flops_per_t(args.gate_grad) * WL.T / (avg_eval_ms / 1000.0) / 1e12
    tc = args.gate_grad == 0 and WL.D <= 32     # the tensor-core kernel runs this workload
    if tc:
        peak, peak_src = tensor_peak_fp32_equiv()
    else:
        peak, peak_src = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
    last = results[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": WL.N, "D": WL.D, "T": WL.T, "step": WL.step,
                   "jac": JAC, "clip": CLIP, "gate_grad": args.gate_grad, "tol": WL.tol,
                   "basis": "eigenvectors of X^T X" if args.basis else "identity",
                   "newton_loop": "CUDA graph, conditional WHILE node (device-side)",
                   "l2": "flushed before every timed step (512 MB write)",
                   "parallelism": f"{world} independent chain(s), one per GPU"},
        "newton_iters": last["iters"], "accept_rate": last["accept_rate"],
        "status": last["status"], "max_residual": last["max_residual"],
        "e2e": {"value": job_value(world, WL.T, e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "tensor" if tc else "alu",
                     "kernel": ("eval_logreg_tc_kernel (evaluate and linearise, tcgen05 3xTF32)"
                                if tc else "eval_logreg_kernel (evaluate and linearise)"),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": EVAL_TRAFFIC_BYTES if tc else None,
                     "peak_source": peak_src + (" x 1.1/2.25 (tf32) / 3 (three products)" if tc else ""),
                     "achieved_is": "algorithmic FP32 flops (10 N D per timestep) / launch time",
                     "avg_launch_ms": avg_eval_ms, "launches": prof["eval_launches"],
                     "timing": "CUDA events around each launch, stream of the launch, "
                               f"{args.steps} profiled solves after the timed region",
                     "scan_avg_ms": prof["scan_ms"] / max(1, prof["scan_launches"])},
        "seq_gpu": None if seq_ms is None else {
            "value": WL.T / (seq_ms / 1000.0), "unit": UNIT, "ms": seq_ms,
            "speedup": (WL.T / (ms / 1000.0)) / (WL.T / (seq_ms / 1000.0))},
        "dense_newton": dense,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# the other configurations (each prints one JSON line of its own)
# ------------------------------------------------------------------------------------------
def _timed(fn, steps, warmup, flush, stream, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms, out = [], None
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms), out


def run_other(args):
    import torch

    import paper_2508_18413_gb300 as P

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    clocks = ClockSampler(0)
    clocks.start()
    line = {"workload": args.workload, "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic", "higher_is_better": True}
    wl = args.workload
    if wl == "c1":
        c = W.C1
        mu, prec, _ = W.gaussian_c1()
        xi, u = W.noise(c.T, 2, seed=0)
        tgt = P.Target("gaussian", 2, mean=torch.tensor(mu, device=dev), prec=torch.tensor(prec, device=dev))
        s0 = torch.zeros(2, dtype=torch.float64, device=dev)
        xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
        opt = P.Options(sampler="mala", step=c.step, jac="dense", precision="f64", atol=c.tol)
        ms, (s, res) = _timed(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), args.steps,
                              args.warmup, flush, stream, torch)
        sms, _ = _timed(lambda: P.pmcmc_seq_solve(tgt, opt, c.T, s0, xid, ud), 1, 1, flush, stream, torch)
        line.update(config=c.name, value=c.T / (ms / 1e3), ms_per_step=ms, newton_iters=res["iters"],
                    status=res["status"], us_per_iter=1e3 * ms / max(1, res["iters"]), dtype="f64",
                    seq_gpu={"value": c.T / (sms / 1e3), "ms": sms, "speedup": sms / ms})
    elif wl in ("c3_diag", "c3_bf16", "c3_block"):
        c = W.C3
        xi, u = W.noise(c.T, 2, seed=0, dtype=np.float32)
        tgt = P.Target("banana", 2)
        s0 = torch.zeros(2, dtype=torch.float32, device=dev)
        xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
        if wl == "c3_block":
            opt = P.Options(sampler="hmc_par_leapfrog", step=c.step, leapfrog_L=c.L, jac="block2",
                            precision="f32", atol=1e-6, rtol=1e-6)
        else:
            opt = P.Options(sampler="hmc", step=c.step, leapfrog_L=c.L, jac="diag", clip=1,
                            precision="f32" if wl == "c3_diag" else "f32_scan_bf16",
                            atol=c.tol, rtol=c.rtol)
        ms, (s, res) = _timed(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), args.steps,
                              args.warmup, flush, stream, torch)
        sopt = P.Options(sampler="hmc", step=c.step, leapfrog_L=c.L, precision="f32")
        sms, _ = _timed(lambda: P.pmcmc_seq_solve(tgt, sopt, c.T, s0, xid, ud), 1, 1, flush, stream, torch)
        line.update(config=f"{c.name} {wl}", value=c.T / (ms / 1e3), ms_per_step=ms,
                    newton_iters=res["iters"], status=res["status"], accept_rate=res["accept_rate"],
                    dtype="f32", seq_gpu={"value": c.T / (sms / 1e3), "ms": sms, "speedup": sms / ms})
    elif wl == "c3_paper":
        # the banana target with the paper's own HMC setting for its Figure 1 example (App. B.4:
        # L = 8, step 0.5, the dense Newton Jacobian scaled by 0.5 and clipped to [-1, 1])
        c = W.C3
        xi, u = W.noise(c.T, 2, seed=0, dtype=np.float32)
        tgt = P.Target("banana", 2)
        s0 = torch.zeros(2, dtype=torch.float32, device=dev)
        xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
        opt = P.Options(sampler="hmc", step=0.5, leapfrog_L=8, jac="dense", damping=0.5, clip=1,
                        precision="f32", atol=c.tol, rtol=c.rtol)
        ms, (s, res) = _timed(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), args.steps,
                              args.warmup, flush, stream, torch)
        sopt = P.Options(sampler="hmc", step=0.5, leapfrog_L=8, precision="f32")
        sms, (sq, _) = _timed(lambda: P.pmcmc_seq_solve(tgt, sopt, c.T, s0, xid, ud), 1, 1, flush,
                              stream, torch)
        dev_max = float(((s - sq).abs() / (1 + sq.abs())).max().item())
        line.update(config="hmc_banana_l8_step0.5_t100000 dense damping 0.5 clip", value=c.T / (ms / 1e3),
                    ms_per_step=ms, newton_iters=res["iters"], status=res["status"],
                    accept_rate=res["accept_rate"], dtype="f32",
                    max_rel_dev_from_sequential=dev_max,
                    seq_gpu={"value": c.T / (sms / 1e3), "ms": sms, "speedup": sms / ms})
    elif wl in ("gibbs_diag", "gibbs_dense"):
        c = W.GIBBS
        S = (c.D - 2) // 2
        X = W.schools_data(S, c.N, seed=0, dtype=np.float32)
        xi = W.gibbs_noise(c.T, S, c.N, seed=1, dtype=np.float32)
        tgt = P.Target("schools", c.D, X=torch.tensor(X, device=dev))
        s0 = torch.tensor(W.schools_init(X), dtype=torch.float32, device=dev)
        xid = torch.tensor(xi, device=dev)
        ud = torch.full((c.T,), 0.5, dtype=torch.float64, device=dev)
        opt = P.Options(sampler="gibbs", jac="diag" if wl == "gibbs_diag" else "dense",
                        precision="f32", atol=c.tol, rtol=c.rtol)
        ms, (s, res) = _timed(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), args.steps,
                              args.warmup, flush, stream, torch)
        sopt = P.Options(sampler="gibbs", precision="f32")
        sms, (sq, _) = _timed(lambda: P.pmcmc_seq_solve(tgt, sopt, c.T, s0, xid, ud), 1, 1, flush,
                              stream, torch)
        dev_max = float(((s - sq).abs() / (1 + sq.abs())).max().item())
        line.update(config=f"{c.name} {wl}", value=c.T / (ms / 1e3), ms_per_step=ms,
                    newton_iters=res["iters"], status=res["status"], dtype="f32",
                    max_rel_dev_from_sequential=dev_max,
                    seq_gpu={"value": c.T / (sms / 1e3), "ms": sms, "speedup": sms / ms})
    elif wl == "adjoint_small":
        # the adjoint workload's shapes (N=5000, D=100) on a 600-step chain: a case small enough
        # for a profiler capture of the tensor-core Jacobian kernel
        c = W.C4
        T = 600
        X, y, _ = W.blr_data(c.N, c.D, seed=0, dtype=np.float32)
        xi, u = W.noise(T, c.D, seed=0, dtype=np.float32)
        tgt = P.Target("logreg", c.D, X=torch.tensor(X, device=dev), y=torch.tensor(y, device=dev))
        s0 = torch.zeros(c.D, dtype=torch.float32, device=dev)
        xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
        sopt = P.Options(sampler="mala", step=c.step, precision="f32")
        s, _ = P.pmcmc_seq_solve(tgt, sopt, T, s0, xid, ud)
        _, _, acc, _ = P.pmcmc_linearize(tgt, P.Options(sampler="mala", step=c.step, jac="zero",
                                                        precision="f32"), T, s0, s, xid, ud,
                                         want_jac=False)
        dL = (2.0 * s / T).contiguous()
        ams, g = _timed(lambda: P.pmcmc_adjoint(tgt, sopt, T, s0, s, acc, xid, ud, dL),
                        args.steps, args.warmup, flush, stream, torch)
        line.update(config=f"mala_logreg_n{c.N}_d{c.D}_t{T} adjoint", value=T / (ams / 1e3),
                    ms_per_step=ams, adjoint={"ms": ams, "grad": g, "accepted": int(acc.sum().item())},
                    dtype="f32")
    elif wl == "c4":
        c = W.C4
        X, y, _ = W.blr_data(c.N, c.D, seed=0, dtype=np.float32)
        xi, u = W.noise(c.T, c.D, seed=0, dtype=np.float32)
        _, Qh = np.linalg.eigh(X.astype(np.float64).T @ X.astype(np.float64))
        tgt = P.Target("logreg", c.D, X=torch.tensor(X, device=dev), y=torch.tensor(y, device=dev),
                       Q=torch.tensor(Qh.astype(np.float32), device=dev))
        s0 = torch.zeros(c.D, dtype=torch.float32, device=dev)
        xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
        opt = P.Options(sampler="mala", step=c.step, jac="diag", precision="f32", atol=c.tol, clip=1,
                        gate_grad=0)
        # The adjoint is taken at the chain's fixed point.  On this workload quasi-Newton needs
        # about 11,000 iterations, so the fixed point comes from the sequential GPU loop; one
        # evaluate pass confirms it (max residual).
        sopt = P.Options(sampler="mala", step=c.step, precision="f32")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s, _ = P.pmcmc_seq_solve(tgt, sopt, c.T, s0, xid, ud)
        e1.record(stream)
        e1.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        f, _, acc, _ = P.pmcmc_linearize(tgt, P.Options(sampler="mala", step=c.step, jac="zero",
                                                        precision="f32"), c.T, s0, s, xid, ud,
                                         want_jac=False)
        fp_res = float((f - s).abs().max().item())
        res = {"accept_rate": float(acc.float().mean().item())}
        dL = (2.0 * s / c.T).contiguous()
        ams, g = _timed(lambda: P.pmcmc_adjoint(tgt, opt, c.T, s0, s, acc, xid, ud, dL),
                        args.steps, 1, flush, stream, torch)
        budget = 256 * 1024 * 1024
        bms, gb = _timed(lambda: P.pmcmc_adjoint(tgt, opt, c.T, s0, s, acc, xid, ud, dL, budget),
                         1, 0, flush, stream, torch)
        # the same adjoint with the J's formed on the CUDA cores (comparison)
        sopt2 = P.Options(sampler="mala", step=c.step, jac="diag", precision="f32", atol=c.tol,
                          clip=1, gate_grad=0, engine="simt")
        cms, gc = _timed(lambda: P.pmcmc_adjoint(tgt, sopt2, c.T, s0, s, acc, xid, ud, dL),
                         1, 0, flush, stream, torch)
        line.update(config=c.name, forward={"ms": fwd_ms, "how": "sequential GPU loop",
                                            "fixed_point_max_residual": fp_res,
                                            "accept_rate": res["accept_rate"],
                                            "value": c.T / (fwd_ms / 1e3)},
                    adjoint={"ms": ams, "grad": g, "accepted": int(acc.sum().item())},
                    adjoint_recompute={"ms": bms, "grad": gb, "jac_budget_bytes": budget},
                    adjoint_cuda_cores={"ms": cms, "grad": gc,
                                        "how": "J formed by the CUDA-core kernel (engine simt)"},
                    value=c.T / ((fwd_ms + ams) / 1e3), ms_per_step=fwd_ms + ams, dtype="f32")
    elif wl == "c5":
        chains = W.batched_mix(512)
        descs = []
        total = 0
        for ch in chains:
            xi, u = W.noise(ch.T, ch.D, seed=ch.noise_seed, dtype=np.float32)
            if ch.target == "gaussian":
                _, Qh = np.linalg.eigh(ch.prec)
                tg = P.Target("gaussian", ch.D, mean=torch.tensor(ch.mu, dtype=torch.float32, device=dev),
                              prec=torch.tensor(ch.prec, dtype=torch.float32, device=dev),
                              Q=torch.tensor(Qh, dtype=torch.float32, device=dev))
            else:
                _, Qh = np.linalg.eigh(ch.X.T @ ch.X)
                tg = P.Target("logreg", ch.D, X=torch.tensor(ch.X, dtype=torch.float32, device=dev),
                              y=torch.tensor(ch.y, dtype=torch.float32, device=dev),
                              Q=torch.tensor(Qh, dtype=torch.float32, device=dev))
            descs.append(P.ChainDesc(tg, ch.sampler, ch.step, ch.L, ch.T,
                                     torch.zeros(ch.D, dtype=torch.float32, device=dev),
                                     torch.tensor(xi, device=dev), torch.tensor(u, device=dev),
                                     torch.empty((ch.T, ch.D), dtype=torch.float32, device=dev)))
            total += ch.T
        opt = P.Options(jac="diag", precision="f32_scan_bf16", atol=1e-5, rtol=1e-5, clip=1,
                        seq_after=args.c5_seq_after)
        ms, res = _timed(lambda: P.pmcmc_solve_batched(descs, opt), args.steps, args.warmup,
                         flush, stream, torch)
        iters = [r["iters"] for r in res]
        n_seq = sum(r["sequential"] for r in res)
        # sequential GPU loop: the chains one after another would take sum of their times; run
        # each chain's sequential kernel on its own stream so they overlap on the device
        streams = [torch.cuda.Stream() for _ in range(16)]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, d in enumerate(descs):
            st = streams[i % len(streams)]
            st.wait_event(e0)
            with torch.cuda.stream(st):
                so = P.Options(sampler=d.sampler, step=d.step, leapfrog_L=d.leapfrog_L, precision="f32")
                P.pmcmc_seq_solve(d.target, so, d.T, d.s0, d.xi, d.u)
        for st in streams:
            stream.wait_stream(st)
        e1.record(stream)
        e1.synchronize()
        sms = e0.elapsed_time(e1)
        line.update(config="512 mixed chains (MALA/HMC L=8, D in {2,8,32}, Gaussian/logistic N=500, "
                           "T~U[1024,65536]), bfloat16 pairs, eigenbasis of P or X^T X per chain",
                    value=total / (ms / 1e3), ms_per_step=ms,
                    samples=total, newton_iters={"max": max(iters), "mean": statistics.mean(iters)},
                    seq_after=args.c5_seq_after, chains_completed_sequentially=n_seq,
                    converged=sum(r["status"] == "OK" for r in res), dtype="f32",
                    seq_gpu={"value": total / (sms / 1e3), "ms": sms, "speedup": sms / ms,
                             "how": "one sequential kernel per chain on 16 streams"})
    elif wl == "scan_sweep":
        rows = []
        peak = _measured_hbm()
        D = args.scan_d
        for prec in args.scan_precisions.split(","):
            Ts = ([int(x) for x in args.scan_t.split(",")] if args.scan_t else
                  [(1 << int(k)) // D for k in args.scan_log2.split(",")])
            for T in Ts:
                n = T * D
                sd = torch.float64 if prec == "f64" else torch.float32
                ad = torch.bfloat16 if prec == "f32_scan_bf16" else sd
                a = (torch.rand((T, D), device=dev) * 1.8 - 0.9).to(ad)
                b = torch.randn((T, D), device=dev).to(ad)
                sv = torch.randn((T, D), device=dev, dtype=sd)
                ms, _ = _timed(lambda: P.pmcmc_scan("diag", prec, a, b, sv), args.steps, args.warmup,
                               flush, stream, torch)
                bytes_ = n * (a.element_size() + sv.element_size()) * 2
                gbs = bytes_ / (ms / 1e3) / 1e9
                rows.append({"precision": prec, "elements": n, "T": T, "D": D, "ms": ms,
                             "GB/s": gbs, "frac_of_measured_hbm": gbs / peak})
                del a, b, sv
        line.update(config=f"diagonal scan alone, a ~ U(-0.9, 0.9), b ~ N(0, 1), D = {D}",
                    unit="GB/s", rows=rows, hbm_peak_measured=peak)
    line["clocks"] = clocks.stop()
    print(json.dumps(line), flush=True)


def _measured_hbm():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        return 6800.0  # fallback figure


def main():
    args = parse()
    if args.scan_kernel:
        os.environ["PMCMC_SCAN_KERNEL"] = "pipe" if args.scan_kernel == "pipe2" else args.scan_kernel
        os.environ["PMCMC_PIPE_CTAS"] = "2" if args.scan_kernel == "pipe2" else "1"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "c2":
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
