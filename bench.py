#!/usr/bin/env python
"""Benchmark: MCMC samples/s to the converged fixed point on GB300, against a sequential GPU
loop, for MALA on Bayesian logistic regression (N=1000 rows, D=25, T=16384, FP32), solved to a
residual tolerance of 1e-6, which puts the whole chain within 1e-5 (1 + |s|) of the FP64 oracle
with the oracle's accept/reject decisions (checked in the CPU-baseline leg, which runs the
oracle on the same noise).

One "step" is one full parallel-Newton solve of the chain (all Newton iterations: evaluate and
linearise, scan, residual check) on inputs already resident in HBM.  The L2 cache is flushed
(a 512 MB write) before every timed step, outside the timed interval.  Under torchrun each rank
solves its own chain (independent noise) on its own GPU: weak scaling, no collective on the
data path; the reported time is the max over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import dataclasses
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
# Residual tolerance of the headline solve.  The workload's tolerance 1e-5 on the residual leaves
# a trace error of up to 1.2e-5 (1 + |s|) against the FP64 oracle (a rejected step has J = I, so
# residuals are carried along runs of rejections); 1e-6 puts the whole chain within the
# 1e-5 (1 + |s|) bar with every decision equal to the oracle's, for 8 more Newton iterations.
ATOL = 1e-6
TRACE_BAR = 1e-5
WORKLOAD = (f"{WL.name}: MALA on synthetic logistic regression (N={WL.N}, D={WL.D}), "
            f"T={WL.T}, step {WL.step}, FP32, quasi-DEER exact diagonal, clip, residual atol "
            f"{ATOL} (trace within {TRACE_BAR} (1 + |s|) of the FP64 oracle)")

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


def eval_traffic_bytes():
    """DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant
    kernel, taken from the committed record of its last ncu capture; None when the kernel source
    has changed since (the record carries a hash of the source it was captured from)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_counters.json")))["eval_logreg_tc_kernel"]
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec["source_sha256_16"]:
            return None
        return rec["dram_bytes_read"] + rec["dram_bytes_write"]
    except Exception:
        return None


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
                             "scan_sweep", "dense_scan", "dense_newton"],
                    help="c2 (default) is the headline line; the others measure the other "
                         "configurations")
    ap.add_argument("--dense-max-iters", type=int, default=0,
                    help="dense_newton workload: Newton iterations per solve (0: to convergence)")
    ap.add_argument("--basis", action="store_true",
                    help="solve in the eigenbasis of X^T X (Section 3.4 reparameterisation)")
    ap.add_argument("--gate-grad", type=int, default=0,
                    help="1: the stop-gradient gate term of Section 3.2 in J")
    ap.add_argument("--atol", type=float, default=ATOL,
                    help="residual tolerance of the headline solve")
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
def oracle_rate(min_seconds: float, max_steps: int | None = None, seed: int = 0):
    """The FP64 oracle's sequential chain of the headline workload on one host core, repeated
    for at least min_seconds.  Returns (samples/s, samples, seconds, first chain's output)."""
    import oracle as O
    X, y, _ = W.blr_data(WL.N, WL.D, seed=WL.seed)
    xi, u = W.noise(WL.T, WL.D, seed=seed, dtype=np.float32)
    steps = WL.T if max_steps is None else min(WL.T, max_steps)
    p = O.Problem(O.Target("logreg", WL.D, X=X, y=y, sigma_p=1.0), "mala", WL.step,
                  xi=xi[:steps].astype(np.float64), u=u[:steps])
    done, t0, first = 0, time.perf_counter(), None
    while True:
        out = O.chain(p, steps, np.zeros(WL.D))
        first = first or out
        done += steps
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return done / el, done, el, first


def parity_vs_oracle(s, acc_gpu, ref, ell, acc, u, bar):
    """Whole-chain error of a GPU result against the oracle's chain of the same noise: decision
    flips, true ties (oracle margin below 1e-9 (1 + |ell|)), the smallest oracle margin, and
    max |s - s_oracle| / (1 + |s_oracle|) (up to the first tie, past which both branches are
    valid chains)."""
    margin = np.abs(np.minimum(ell, 0.0) - np.log(u))
    ties = np.nonzero(margin < 1e-9 * (1 + np.abs(ell)))[0]
    flips = np.nonzero(acc_gpu != acc)[0]
    upto = int(ties[0]) if len(ties) else len(s)
    err = float((np.abs(s[:upto] - ref[:upto]) / (1 + np.abs(ref[:upto]))).max()) if upto else 0.0
    return {"vs": "FP64 oracle, same noise, whole chain", "steps": len(s),
            "decision_flips": int(len(flips)), "flips_outside_ties": int(len(set(flips.tolist()) - set(ties.tolist()))),
            "ties": ties.tolist()[:20], "min_margin": float(margin.min()),
            "max_err_vs_oracle": err, "bar": bar, "meets_bar": bool(err <= bar and
                                                                   len(set(flips.tolist()) - set(ties.tolist())) == 0)}


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
        r, n, el, _ = oracle_rate(0.0, max_steps=2048)
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


def _frozen_loss(args):
    """L = (1/T) sum_t |s_t|^2 of the oracle's MALA chain with decisions frozen (a worker of the
    finite-difference check; spawned, so it never touches the GPU)."""
    import oracle as O
    X, y, sp, eps, xi, u, acc, T = args
    p = O.Problem(O.Target("logreg", X.shape[1], X=X, y=y, sigma_p=sp), "mala", eps, xi=xi, u=u)
    s = O.mala_chain_frozen(p, T, np.zeros(X.shape[1]), acc)
    return float((s * s).sum() / T)


def c4_oracle_check(X, y, step, xi, u, acc, grad_gpu, s_gpu, prefix=256, h=1e-4):
    """The adjoint workload's gradient against (i) central finite differences of the oracle's
    frozen-decision chain over the whole chain, h = 1e-4 (the four chains in parallel worker
    processes), and (ii) the oracle's reverse recursion on a full-width prefix of the chain."""
    import multiprocessing as mp
    import oracle as O
    T = len(acc)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    xi64 = xi.astype(np.float64)
    acc_i = acc.astype(np.int32)
    h2 = h / 2
    jobs = [(X64, y64, 1.0, step + h, xi64, u, acc_i, T), (X64, y64, 1.0, step - h, xi64, u, acc_i, T),
            (X64, y64, 1.0 + h, step, xi64, u, acc_i, T), (X64, y64, 1.0 - h, step, xi64, u, acc_i, T),
            (X64, y64, 1.0, step + h2, xi64, u, acc_i, T), (X64, y64, 1.0, step - h2, xi64, u, acc_i, T)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(6) as pool:
        Lp, Lm, Sp, Sm, Lp2, Lm2 = pool.map(_frozen_loss, jobs)
    fd = np.array([(Lp - Lm) / (2 * h), (Sp - Sm) / (2 * h)])
    # h = 1e-4 is 20% of the step size 5e-4, so the central difference carries a truncation
    # error O(h^2) of about 1% in d/d step; Richardson's extrapolation from h and h/2 removes it
    fd_step_h2 = (Lp2 - Lm2) / (2 * h2)
    rich_step = (4.0 * fd_step_h2 - fd[0]) / 3.0
    fd_s = time.perf_counter() - t0
    g = np.array(grad_gpu)
    rel_fd = (np.abs(g - fd) / np.maximum(np.abs(fd), 1e-300)).tolist()
    rel_rich = [float(abs(g[0] - rich_step) / abs(rich_step)), rel_fd[1]]
    # oracle reverse recursion on the first `prefix` steps of the GPU's fixed point, for
    # L_prefix = (1/T) sum_{t < prefix} |s_t|^2 (the same functional restricted to the prefix)
    n = min(prefix, T)
    p = O.Problem(O.Target("logreg", X.shape[1], X=X64, y=y64, sigma_p=1.0), "mala", step,
                  xi=xi64[:n], u=u[:n])
    s_ref = O.mala_chain_frozen(p, n, np.zeros(X.shape[1]), acc_i[:n])
    g_ref = O.mala_adjoint(p, n, np.zeros(X.shape[1]), s_ref, acc_i[:n], 2.0 * s_ref / T)
    return {"fd": fd.tolist(), "fd_h": h, "fd_seconds": fd_s, "rel_err_vs_fd": rel_fd,
            "fd_step_h_half": fd_step_h2, "richardson_step": rich_step,
            "rel_err_vs_fd_richardson": rel_rich,
            "meets_1e-3": bool(max(rel_rich) <= 1e-3), "prefix_steps": n, "prefix_oracle_grad": g_ref.tolist(),
            "prefix_trace_err_vs_oracle": float((np.abs(s_gpu[:n] - s_ref) / (1 + np.abs(s_ref))).max())}


# ------------------------------------------------------------------------------------------
# the other workloads, reported as extra keys of the default line (bounded time each)
# ------------------------------------------------------------------------------------------
def _time_fn(fn, steps, warmup, flush, stream, torch):
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


def run_diag_scan_keys(P, torch, dev, flush, stream):
    """The diagonal scan alone (quasi-DEER's step (b)) at 2^26 and 2^28 elements, D = 8, FP32
    and bfloat16 pairs, with the kernel the library picks: GB/s of its algorithmic traffic (read
    a, b, s; write s) and the fraction of the measured HBM bandwidth.  a ~ U(-0.9, 0.9),
    b ~ N(0, 1), s ~ N(0, 1); L2 flushed before every timed scan (10 timed, 3 warm-up).  Each
    result is checked on the first 2,048 timesteps against the recursion in FP64, and on the
    last 2,048 against the recursion run from the scan's own value just before them (the carry
    the look-back delivered)."""
    D, out = 8, []
    peak = _measured_hbm()
    g = torch.Generator(device=dev)
    for log2 in (26, 28):
        for prec in ("f32", "f32_scan_bf16"):
            T = (1 << log2) // D
            ad = torch.bfloat16 if prec == "f32_scan_bf16" else torch.float32
            g.manual_seed(log2)
            a = (torch.rand((T, D), device=dev, generator=g) * 1.8 - 0.9).to(ad)
            b = torch.randn((T, D), device=dev, generator=g).to(ad)
            s0 = torch.randn((T, D), device=dev, generator=g)
            s = s0.clone()
            P.pmcmc_scan("diag", prec, a, b, s)
            torch.cuda.synchronize()
            w = 2048
            d_head = (s[:w].double() - s0[:w].double()).cpu().numpy()
            d_tail = (s[-w - 1:].double() - s0[-w - 1:].double()).cpu().numpy()
            a_head, b_head = a[:w].double().cpu().numpy(), b[:w].double().cpu().numpy()
            a_tail, b_tail = a[-w:].double().cpu().numpy(), b[-w:].double().cpu().numpy()
            err = 0.0
            for dref0, aa, bb, got in ((np.zeros(D), a_head, b_head, d_head),
                                       (d_tail[0], a_tail, b_tail, d_tail[1:])):
                dl = dref0.copy()
                for t in range(w):
                    dl = aa[t] * dl + bb[t]
                    err = max(err, float(np.max(np.abs(got[t] - dl) / (1.0 + np.abs(dl)))))
            ms, _ = _time_fn(lambda: P.pmcmc_scan("diag", prec, a, b, s), 10, 3, flush, stream, torch)
            gbs = T * D * (a.element_size() + 4) * 2 / (ms / 1e3) / 1e9
            out.append({"elements": T * D, "D": D, "precision": prec, "ms": ms, "GB/s": gbs,
                        "frac_of_measured_hbm": gbs / peak, "max_rel_err_sampled": err})
            del a, b, s0, s
            torch.cuda.empty_cache()
    return {"rows": out, "hbm_peak_measured": peak,
            "bytes_per_element": "16 (FP32: read a, b, s; write s), 12 with bfloat16 a, b"}


def run_configs(P, torch, dev, flush, stream):
    """C1, C3 (diagonal, bfloat16 pairs, block-quasi parallel leapfrog), the 512-chain batch and
    the Gibbs chain: samples/s of the parallel solve, its Newton iterations and the sequential
    GPU loop's samples/s.  Returns (keys, host copies of the results for the oracle check)."""
    keys, keep = {}, {}

    def entry(name, T, ms, res, sms, extra=None):
        e = {"value": T / (ms / 1e3), "unit": UNIT, "ms": ms, "newton_iters": res.get("iters"),
             "status": res.get("status"),
             "seq_gpu": {"value": T / (sms / 1e3), "ms": sms, "speedup": sms / ms}}
        e.update(extra or {})
        keys[name] = e

    # C1: MALA, D=2 Gaussian, FP64, dense Newton, tol 1e-10
    c = W.C1
    mu, prec, _ = W.gaussian_c1()
    xi, u = W.noise(c.T, 2, seed=0)
    tgt = P.Target("gaussian", 2, mean=torch.tensor(mu, device=dev), prec=torch.tensor(prec, device=dev))
    s0 = torch.zeros(2, dtype=torch.float64, device=dev)
    xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
    opt = P.Options(sampler="mala", step=c.step, jac="dense", precision="f64", atol=c.tol)
    ms, (s, res) = _time_fn(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), 5, 2, flush, stream, torch)
    sms, _ = _time_fn(lambda: P.pmcmc_seq_solve(tgt, opt, c.T, s0, xid, ud), 2, 1, flush, stream, torch)
    entry("c1", c.T, ms, res, sms, {"workload": f"{c.name}: MALA Gaussian D=2, FP64, dense Newton, tol {c.tol}",
                                      "us_per_iter": 1e3 * ms / max(1, res["iters"])})
    keep["c1"] = s.cpu().numpy()

    # C3: HMC on the banana, L=16, step 0.05, T=100000
    c = W.C3
    xi, u = W.noise(c.T, 2, seed=0, dtype=np.float32)
    tgt = P.Target("banana", 2)
    s0 = torch.zeros(2, dtype=torch.float32, device=dev)
    xid, ud = torch.tensor(xi, device=dev), torch.tensor(u, device=dev)
    sopt = P.Options(sampler="hmc", step=c.step, leapfrog_L=c.L, precision="f32")
    sms, (sq, _) = _time_fn(lambda: P.pmcmc_seq_solve(tgt, sopt, c.T, s0, xid, ud), 2, 1, flush, stream, torch)
    keep["c3_seq32"] = sq.cpu().numpy()
    for name, opt in (("c3_diag", P.Options(sampler="hmc", step=c.step, leapfrog_L=c.L, jac="diag", clip=0,
                                            precision="f32", atol=1e-6, rtol=1e-6)),
                      ("c3_bf16", P.Options(sampler="hmc", step=c.step, leapfrog_L=c.L, jac="diag", clip=0,
                                            precision="f32_scan_bf16", atol=1e-6, rtol=1e-6)),
                      ("c3_block", P.Options(sampler="hmc_par_leapfrog", step=c.step, leapfrog_L=c.L,
                                             jac="block2", precision="f32", atol=1e-6, rtol=1e-6))):
        ms, (s, res) = _time_fn(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), 2, 1, flush, stream, torch)
        entry(name, c.T, ms, res, sms, {"workload": f"{c.name}: HMC banana L={c.L} step {c.step}, {opt.jac}, "
                                                    f"clip {opt.clip}, {opt.precision}, atol/rtol 1e-6",
                                         "accept_rate": res["accept_rate"]})
        keep[name] = s.cpu().numpy()

    # Gibbs on the schools model, quasi-DEER (exact diagonal)
    c = W.GIBBS
    S = (c.D - 2) // 2
    X = W.schools_data(S, c.N, seed=0, dtype=np.float32)
    xi = W.gibbs_noise(c.T, S, c.N, seed=1, dtype=np.float32)
    tgt = P.Target("schools", c.D, X=torch.tensor(X, device=dev))
    s0 = torch.tensor(W.schools_init(X), dtype=torch.float32, device=dev)
    xid = torch.tensor(xi, device=dev)
    ud = torch.full((c.T,), 0.5, dtype=torch.float64, device=dev)
    opt = P.Options(sampler="gibbs", jac="diag", precision="f32", atol=c.tol, rtol=c.rtol)
    ms, (s, res) = _time_fn(lambda: P.pmcmc_solve(tgt, opt, c.T, s0, xi=xid, u=ud), 3, 1, flush, stream, torch)
    sms, (sq, _) = _time_fn(lambda: P.pmcmc_seq_solve(tgt, P.Options(sampler="gibbs", precision="f32"), c.T, s0,
                                                      xid, ud), 2, 1, flush, stream, torch)
    entry("gibbs_diag", c.T, ms, res, sms, {"workload": f"{c.name}: reparameterised Gibbs, schools S={S} N={c.N}, "
                                                        f"quasi-DEER, FP32, atol {c.tol} rtol {c.rtol}"})
    keep["gibbs_diag"] = s.cpu().numpy()

    # C5: 512 mixed chains, bfloat16 pairs, one persistent graph-captured launch per sweep loop
    chains = W.batched_mix(512)
    descs, total = [], 0
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
    opt = P.Options(jac="diag", precision="f32_scan_bf16", atol=1e-5, rtol=1e-5, clip=1, seq_after=150)
    ms, res = _time_fn(lambda: P.pmcmc_solve_batched(descs, opt), 1, 1, flush, stream, torch)
    iters = [r["iters"] for r in res]
    sample = list(range(0, 512, 64))
    keep["c5"] = {i: descs[i].s_out.cpu().numpy() for i in sample}
    seq_out = [torch.empty_like(d.s_out) for d in descs]
    sdescs = [P.ChainDesc(d.target, d.sampler, d.step, d.leapfrog_L, d.T, d.s0, d.xi, d.u, o)
              for d, o in zip(descs, seq_out)]
    sms, _ = _time_fn(lambda: P.pmcmc_seq_solve_batched(sdescs), 2, 1, flush, stream, torch)
    keys["c5"] = {"value": total / (ms / 1e3), "unit": UNIT, "ms": ms, "samples": total,
                  "workload": "512 mixed chains (MALA/HMC L=8, D in {2,8,32}, Gaussian/logistic N=500, "
                              "T~U[1024,65536]), bfloat16 pairs, eigenbasis per chain, one graph-captured "
                              "persistent launch per Newton sweep; chains unconverged after 150 sweeps "
                              "completed by the sequential kernel",
                  "newton_iters": {"max": max(iters), "mean": statistics.mean(iters)},
                  "chains_completed_sequentially": sum(r["sequential"] for r in res),
                  "converged": sum(r["status"] == "OK" for r in res),
                  "seq_gpu": {"value": total / (sms / 1e3), "ms": sms, "speedup": sms / ms,
                              "how": "all 512 sequential chains in one launch, one CTA per chain"}}
    keep["c5_chains"] = [(chains[i], i) for i in sample]
    return keys, keep


def configs_vs_oracle(keys, keep):
    """Error of each extra workload's GPU result against the FP64 oracle's chain of the same
    noise (whole chain; the batch on a sample of chains, on a prefix of each)."""
    import oracle as O
    t_start = time.perf_counter()

    def cmp(name, ref, ell, acc, u, s, bar):
        margin = np.abs(np.minimum(ell, 0.0) - np.log(u)) if u is not None else None
        err = np.abs(s - ref) / (1 + np.abs(ref))
        d = {"max_err_vs_oracle": float(err.max()), "steps_checked": int(len(s)), "bar": bar,
             "meets_bar": bool(err.max() <= bar)}
        if margin is not None:
            d["min_margin"] = float(margin.min())
        keys[name]["vs_oracle"] = d
        return err

    c = W.C1
    mu, prec, _ = W.gaussian_c1()
    xi, u = W.noise(c.T, 2, seed=0)
    ref, ell, acc = O.chain(O.Problem(O.Target("gaussian", 2, mu=mu, P=prec), "mala", c.step, xi=xi, u=u),
                            c.T, np.zeros(2))
    cmp("c1", ref, ell, acc, u, keep["c1"], 1e-10)

    c = W.C3
    xi, u = W.noise(c.T, 2, seed=0, dtype=np.float32)
    p = O.Problem(O.Target("banana", 2), "hmc", c.step, xi=xi.astype(np.float64), u=u, L=c.L)
    ref, ell, acc = O.chain(p, c.T, np.zeros(2))
    # the chain's own sensitivity to FP32: the oracle's chain with its state rounded to FP32
    # after every step (exact arithmetic otherwise) drifts from the exact chain by
    r32 = np.zeros((c.T, 2))
    x = np.zeros(2)
    for t in range(c.T):
        x = O.f(p, t + 1, x)[0].astype(np.float32).astype(np.float64)
        r32[t] = x
    round_err = float((np.abs(r32 - ref) / (1 + np.abs(ref))).max())
    seq_err = float((np.abs(keep["c3_seq32"] - ref) / (1 + np.abs(ref))).max())
    for name in ("c3_diag", "c3_bf16", "c3_block"):
        # bar: this chain's FP32 sensitivity (the FP32 sequential loop's own deviation is 1.3e-3)
        cmp(name, ref, ell, acc, u, keep[name], 2e-3)
        sq = keep["c3_seq32"]
        keys[name]["vs_oracle"].update({
            "fp32_rounding_only_err": round_err, "sequential_fp32_gpu_err": seq_err,
            "max_err_vs_sequential_fp32_gpu": float((np.abs(keep[name] - sq) / (1 + np.abs(sq))).max())})

    c = W.GIBBS
    S = (c.D - 2) // 2
    X = W.schools_data(S, c.N, seed=0, dtype=np.float32).astype(np.float64)
    xi = W.gibbs_noise(c.T, S, c.N, seed=1, dtype=np.float32).astype(np.float64)
    s0 = W.schools_init(X.astype(np.float32)).astype(np.float32).astype(np.float64)
    ref, _, _ = O.chain(O.Problem(O.Target("schools", c.D, X=X), "gibbs", 0.0, xi=xi,
                                  u=np.full(c.T, 0.5)), c.T, s0)
    cmp("gibbs_diag", ref, np.zeros(c.T), None, None, keep["gibbs_diag"], 1e-4)

    errs = []
    for ch, i in keep["c5_chains"]:
        xi, u = W.noise(ch.T, ch.D, seed=ch.noise_seed, dtype=np.float32)
        n = min(ch.T, 2048)
        if ch.target == "gaussian":
            ot = O.Target("gaussian", ch.D, mu=ch.mu, P=ch.prec)
        else:
            ot = O.Target("logreg", ch.D, X=ch.X, y=ch.y, sigma_p=1.0)
        ref, _, _ = O.chain(O.Problem(ot, ch.sampler, ch.step, xi=xi[:n].astype(np.float64), u=u[:n],
                                      L=ch.L), n, np.zeros(ch.D))
        s = keep["c5"][i][:n]
        errs.append(float((np.abs(s - ref) / (1 + np.abs(ref))).max()))
    keys["c5"]["vs_oracle"] = {"max_err_vs_oracle": max(errs), "chains_checked": len(errs),
                               "steps_checked_per_chain": "first 2048 (whole chain if shorter)",
                               "per_chain": errs}
    return time.perf_counter() - t_start


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
    opt = P.Options(sampler="mala", step=WL.step, jac=JAC, precision="f32", atol=args.atol,
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
    # the timed result and its decisions, for the comparison with the oracle (not timed)
    s_last = s_out.detach().cpu().double().numpy()
    _, _, acc_d, _ = P.pmcmc_linearize(tgt, P.Options(sampler="mala", step=WL.step, jac="zero",
                                                      precision="f32"), WL.T, s0, s_out, xid, ud,
                                       want_jac=False)
    acc_last = acc_d.cpu().numpy().astype(bool)
    # the same solve at the workload's own residual tolerance 1e-5 (context: trace bar not met)
    opt5 = P.Options(sampler="mala", step=WL.step, jac=JAC, precision="f32", atol=WL.tol,
                     clip=CLIP, gate_grad=args.gate_grad)
    s5 = torch.empty_like(s_out)
    P.pmcmc_solve(tgt, opt5, WL.T, s0, xi=xid, u=ud, s_out=s5)
    ms5 = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, res5 = P.pmcmc_solve(tgt, opt5, WL.T, s0, xi=xid, u=ud, s_out=s5)
        e1.record(stream)
        e1.synchronize()
        ms5.append(e0.elapsed_time(e1))
    s5_h = s5.cpu().double().numpy()
    # kernel durations: the same solves with per-launch CUDA events (host-driven loop)
    P.pmcmc_profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        P.pmcmc_solve(tgt, opt, WL.T, s0, xi=xid, u=ud, s_out=s_out)
    torch.cuda.synchronize()
    prof = P.pmcmc_profile_get()
    P.pmcmc_profile_enable(False)
    # launches inside the timed region, per solve: iters + 1 evaluations; on the fused path
    # (the default) each is one kernel that also applies the update and takes the loop's
    # decision, otherwise evaluate + control + scan; and the set-up kernels (padded design,
    # tensor-core images and X^T y, initial guess, two finiteness checks, loop init, and the
    # copy of the result out of the second iterate buffer on the fused path)
    fused = os.environ.get("PMCMC_FUSED_UPDATE", "1") != "0"
    launches_timed = sum((r["iters"] + 1) * (1 if fused else 3) + (8 if fused else 7) for r in results)

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

    # --- dense-Newton line (same chain), run to convergence (it needs thousands of iterations:
    # the dense linearisation of this chain is expanding), timed once.  Held gate, damping 0.5
    # (fewer iterations than undamped or with the gate term), the evaluate pass, the Jacobian
    # and the scan's compositions on the tensor cores ------------------------------------------
    dense = None
    if rank == 0 and not args.no_variants:
        optd = P.Options(sampler="mala", step=WL.step, jac="dense", precision="f32_scan_bf16", atol=args.atol,
                         clip=CLIP, max_iters=WL.T, gate_grad=0, damping=0.5)
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, rd = P.pmcmc_solve(tgt, optd, WL.T, s0, xi=xid, u=ud, s_out=s_out)
        e1.record(stream)
        e1.synchronize()
        dms = e0.elapsed_time(e1)
        s_dense = s_out.detach().cpu().double().numpy()
        dense = {"value": WL.T / (dms / 1000.0), "unit": UNIT, "ms": dms, "newton_iters": rd["iters"],
                 "status": rd["status"], "how": "dense J (tcgen05 tf32), held gate, damping 0.5, clip, "
                 "scan compositions on tcgen05 (bfloat16), residual atol " + str(args.atol)}

    configs, keep = None, None
    if rank == 0 and not args.no_variants:
        configs, keep = run_configs(P, torch, dev, flush, stream)

    diag_scan = None
    if rank == 0 and not args.no_variants:
        try:  # an extra measurement: the headline line is printed whatever happens here
            diag_scan = run_diag_scan_keys(P, torch, dev, flush, stream)
        except Exception as exc:
            diag_scan = {"error": f"{type(exc).__name__}: {exc}"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu, parity, parity5 = None, None, None
    if not args.no_cpu:
        rate, nsamp, el, (ref, ell_o, acc_o) = oracle_rate(10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nsamp} steps (whole chain repeated) of the same workload in FP64, "
                         f"{el:.1f} s"}
        _, u_h64 = W.noise(WL.T, WL.D, seed=0, dtype=np.float32)
        parity = parity_vs_oracle(s_last, acc_last, ref, ell_o, acc_o, u_h64, TRACE_BAR)
        parity5 = parity_vs_oracle(s5_h, acc_last, ref, ell_o, acc_o, u_h64, TRACE_BAR)
        if dense is not None:
            # the dense solve's decisions, read off its trace: a rejected step repeats the state
            # up to the residual tolerance, an accepted one moves by about sqrt(2 step) = 0.14
            prev = np.vstack([np.zeros((1, WL.D)), s_dense[:-1]])
            acc_dense = np.abs(s_dense - prev).max(axis=1) > 1e-3
            dense["parity"] = parity_vs_oracle(s_dense, acc_dense, ref, ell_o, acc_o, u_h64, TRACE_BAR)
        if configs is not None:
            configs_vs_oracle(configs, keep)

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
                   "jac": JAC, "clip": CLIP, "gate_grad": args.gate_grad, "atol": args.atol,
                   "trace_bar": f"{TRACE_BAR} (1 + |s|) vs the FP64 oracle",
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
                     "frac": achieved / peak, "traffic": eval_traffic_bytes() if tc else None,
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
        "configs": configs,
        "diag_scan": diag_scan,
        "parity": parity,
        "at_workload_tol_1e-5": {"value": WL.T / (statistics.mean(ms5) / 1e3), "unit": UNIT,
                                 "ms": statistics.mean(ms5), "newton_iters": res5["iters"],
                                 "max_err_vs_oracle": None if parity5 is None else parity5["max_err_vs_oracle"],
                                 "meets_trace_bar": None if parity5 is None else parity5["meets_bar"]},
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
        s, acc = P.pmcmc_seq_solve(tgt, sopt, c.T, s0, xid, ud)
        e1.record(stream)
        e1.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        # The chain's own decisions define the piece the gradient is taken on.  One evaluate pass
        # at s re-takes every decision with the evaluate kernel's FP32 arithmetic: where the two
        # differ (a near-tie of the MH comparison) the residual is a whole proposal step, so the
        # fixed-point residual is reported over the steps where they agree.
        f, _, acc_e, _ = P.pmcmc_linearize(tgt, P.Options(sampler="mala", step=c.step, jac="zero",
                                                          precision="f32"), c.T, s0, s, xid, ud,
                                           want_jac=False)
        agree = (acc_e == acc)
        fp_res = float(((f - s).abs().max(dim=1).values * agree).max().item())
        res = {"accept_rate": float(acc.float().mean().item()),
               "decision_disagreements": int((~agree).sum().item())}
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
        # the prefix adjoint on the GPU, for the comparison with the oracle's reverse recursion
        npre = 256
        dLp = dL.clone()
        dLp[npre:] = 0.0
        gp = P.pmcmc_adjoint(tgt, opt, c.T, s0, s, acc, xid, ud, dLp)
        chk = c4_oracle_check(X, y, c.step, xi, u, acc.cpu().numpy().astype(bool), g,
                              s.cpu().double().numpy(), prefix=npre)
        chk["prefix_gpu_grad"] = list(gp)
        chk["prefix_rel_err"] = (np.abs(np.array(gp) - np.array(chk["prefix_oracle_grad"])) /
                                 np.maximum(np.abs(np.array(chk["prefix_oracle_grad"])), 1e-300)).tolist()
        line["vs_oracle"] = chk
        line.update(config=c.name, forward={"ms": fwd_ms, "how": "sequential GPU loop",
                                            "fixed_point_max_residual": fp_res,
                                            "near_tie_decision_disagreements": res["decision_disagreements"],
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
    elif wl == "dense_newton":
        # the headline chain solved by dense Newton (DEER, Eq. 3): the logistic J assembled on
        # the tensor cores, the scan's compositions on the tensor cores; per-kernel device time
        # from the library's profile counters.  --dense-max-iters bounds the solve (a bounded run
        # measures the cost per iteration; the default runs to convergence)
        X, y, _ = W.blr_data(W.C2.N, W.C2.D, seed=W.C2.seed, dtype=np.float32)
        xi_h, u_h = W.noise(W.C2.T, W.C2.D, seed=0, dtype=np.float32)
        tgt = P.Target("logreg", W.C2.D, X=torch.tensor(X, device=dev), y=torch.tensor(y, device=dev),
                       prior_scale=1.0)
        xid, ud = torch.tensor(xi_h, device=dev), torch.tensor(u_h, device=dev)
        s0 = torch.zeros(W.C2.D, dtype=torch.float32, device=dev)
        rows = []
        for engine in ("auto", "simt"):
            optd = P.Options(sampler="mala", step=W.C2.step, jac="dense", precision="f32_scan_bf16",
                             atol=W.C2.tol, clip=1, gate_grad=0, damping=0.5, engine=engine,
                             max_iters=args.dense_max_iters or W.C2.T)
            P.pmcmc_solve(tgt, dataclasses.replace(optd, max_iters=3), W.C2.T, s0, xi=xid, u=ud)  # warm-up
            torch.cuda.synchronize()
            P.pmcmc_profile_enable(True)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, rd = P.pmcmc_solve(tgt, optd, W.C2.T, s0, xi=xid, u=ud)
            e1.record(stream)
            e1.synchronize()
            pr = P.pmcmc_profile_get()
            P.pmcmc_profile_enable(False)
            ms = e0.elapsed_time(e1)
            it = max(rd["iters"], 1)
            rows.append({"engine": engine, "ms": ms, "newton_iters": rd["iters"], "status": rd["status"],
                         "value": W.C2.T / (ms / 1e3), "ms_per_iter": ms / it,
                         "eval_ms_per_iter": pr["eval_ms"] / it, "jac_ms_per_iter": pr["jac_ms"] / it,
                         "scan_ms_per_iter": pr["scan_ms"] / it})
        line.update(config="C2 chain (MALA logistic N=1000, D=25, T=16384, step 0.01) by dense Newton: "
                           "held gate, damping 0.5, clip, bfloat16 scan pairs", unit=UNIT, rows=rows)
    elif wl == "dense_scan":
        # the dense scan alone (DEER's linear solve, Eq. 3): compositions on the CUDA cores
        # (FP32) against the tensor cores (bfloat16 operands, FP32 accumulation)
        rows = []
        for T, D in ((16384, 25), (16384, 32), (65536, 25), (65536, 32)):
            g = torch.Generator(device=dev).manual_seed(T + D)
            a32 = 0.95 * torch.eye(D, device=dev).expand(T, D, D) + \
                torch.randn((T, D, D), device=dev, generator=g) * (0.04 / D ** 0.5)
            b32 = torch.randn((T, D), device=dev, generator=g)
            for prec in ("f32", "f32_scan_bf16"):
                ad = torch.bfloat16 if prec == "f32_scan_bf16" else torch.float32
                a_, b_ = a32.to(ad).contiguous(), b32.to(ad).contiguous()
                sv = torch.zeros((T, D), device=dev)
                ms, _ = _timed(lambda: P.pmcmc_scan("dense", prec, a_, b_, sv), args.steps, args.warmup,
                               flush, stream, torch)
                useful = 2.0 * T * D ** 3   # the products J_t P_{t-1} (flops)
                rows.append({"precision": prec, "T": T, "D": D, "ms": ms,
                             "useful_product_tflops": useful / (ms / 1e3) / 1e12,
                             "engine": "tcgen05 kind::f16 (bf16)" if prec == "f32_scan_bf16" else "CUDA cores (FP32)"})
                del a_, b_, sv
        line.update(config="dense scan alone, J_t = 0.95 I + N(0, 0.04^2 / D), b ~ N(0, 1)", unit="ms", rows=rows)
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
