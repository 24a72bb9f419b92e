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
JAC = "diag"        # quasi-DEER with the exact diagonal
WORKLOAD = (f"{WL.name}: MALA on synthetic logistic regression (N={WL.N}, D={WL.D}), "
            f"T={WL.T}, step {WL.step}, FP32, quasi-DEER exact diagonal, clip, tol {WL.tol}")

# FP32 FMA peak of the GB300 (no tensor cores): 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic flops of one evaluate-and-linearise launch (MALA, exact diagonal, gate term):
# per timestep 2 gradients (2 N D MACs each), diag(X^T W X) (N D), two Hessian-vector products
# (2 N D each) = 9 N D MACs = 18 N D flops.
ALG_FLOPS_PER_T = 18 * WL.N * WL.D
# DRAM traffic of one evaluate-and-linearise launch from the committed ncu capture
# (profiles/eval_logreg_c2.md); None until that capture exists for the current kernel.
EVAL_TRAFFIC_BYTES = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-variants", action="store_true", help="skip the dense-Newton line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
    tgt = P.Target("logreg", WL.D, X=Xd, y=yd, prior_scale=1.0)
    opt = P.Options(sampler="mala", step=WL.step, jac=JAC, precision="f32", atol=WL.tol,
                    clip=CLIP)
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
    P.pmcmc_profile_enable(True)
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
    prof = P.pmcmc_profile_get()
    P.pmcmc_profile_enable(False)
    clk = clocks.stop()

    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        n = torch.tensor([prof["launches"]], device=dev, dtype=torch.float64)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        launches = int(n.item())
    else:
        launches = int(prof["launches"])
    value = world * WL.T / (ms / 1000.0)

    # --- end to end through the public API with host buffers (pinned) ---------------------
    Xh = torch.tensor(X).pin_memory()
    yh = torch.tensor(y).pin_memory()
    xih = torch.tensor(xi_h).pin_memory()
    uh = torch.tensor(u_h).pin_memory()
    s0h = torch.zeros(WL.D, dtype=torch.float32).pin_memory()
    outh = torch.empty((WL.T, WL.D), dtype=torch.float32).pin_memory()
    Xe, ye, xie, ue, s0e = (torch.empty_like(t, device=dev) for t in (Xh, yh, xih, uh, s0h))
    tgt_e = P.Target("logreg", WL.D, X=Xe, y=ye, prior_scale=1.0)
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
    e2e = statistics.mean(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = float(t.item())

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
                         clip=CLIP)
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
    achieved = ALG_FLOPS_PER_T * WL.T / (avg_eval_ms / 1000.0) / 1e12
    last = results[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": WL.N, "D": WL.D, "T": WL.T, "step": WL.step,
                   "jac": JAC, "clip": CLIP, "tol": WL.tol,
                   "l2": "flushed before every timed step (512 MB write)",
                   "parallelism": f"{world} independent chain(s), one per GPU"},
        "newton_iters": last["iters"], "accept_rate": last["accept_rate"],
        "status": last["status"], "max_residual": last["max_residual"],
        "e2e": {"value": world * WL.T / (e2e / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "eval_logreg_kernel (evaluate and linearise)",
                     "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": EVAL_TRAFFIC_BYTES,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "avg_launch_ms": avg_eval_ms, "launches": prof["eval_launches"],
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
