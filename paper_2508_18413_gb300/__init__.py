"""Parallel-Newton MCMC on one GB300 (arXiv 2508.18413), Python binding of libpmcmc.

Every function here has the name of the C entry point it calls (include/pmcmc.h) and only
marshals arguments: torch tensors give device pointers and the current CUDA stream; every step
of the computation runs in the library's CUDA kernels.  There is no CPU fallback: without the
built library or a CUDA device these functions raise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L
from ._lib import ENGINES, JACS, PRECISIONS, SAMPLERS, STATUS_NAMES, TARGETS

__all__ = [
    "PmcmcError", "Target", "Options", "pmcmc_create", "pmcmc_gen_noise", "pmcmc_solve",
    "pmcmc_seq_solve", "pmcmc_linearize", "pmcmc_scan", "pmcmc_adjoint", "pmcmc_solve_batched",
    "pmcmc_solve_async", "result_from_device",
    "ChainDesc", "real_dtype", "loaded_library_path", "pmcmc_profile_enable",
    "pmcmc_profile_get", "pmcmc_scan_noalloc", "pmcmc_scan_plan", "ChainSolve", "solve_differentiable",
    "pmcmc_seq_solve_batched",
]


class PmcmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def real_dtype(precision: str) -> torch.dtype:
    return torch.float64 if precision == "f64" else torch.float32


def loaded_library_path() -> str:
    return L.LIB_PATH


_contexts: dict[int, int] = {}


def pmcmc_create(device: int | None = None) -> int:
    """Return the (cached) library context of a CUDA device."""
    lib = L.load()
    if not torch.cuda.is_available():
        raise PmcmcError(L.PMCMC_EINVAL, "no CUDA device: the library has no CPU path")
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _contexts:
        h = C.c_void_p()
        st = lib.pmcmc_create(C.byref(h), dev)
        if st != 0:
            raise PmcmcError(st, "pmcmc_create failed")
        _contexts[dev] = h.value
    return _contexts[dev]


def _check(ctx, st, allow_not_converged=True):
    if st == 0 or (allow_not_converged and st == L.PMCMC_NOT_CONVERGED):
        return st
    msg = L.load().pmcmc_last_error(ctx)
    raise PmcmcError(st, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


@dataclass
class Target:
    """A built-in target (include/pmcmc.h pmcmc_target); tensors live on the GPU.

    kind "schools": X holds the S x N scores of the hierarchical Gaussian model sampled by the
    "gibbs" sampler, D = 2 + 2 S."""
    kind: str
    D: int
    mean: torch.Tensor | None = None
    prec: torch.Tensor | None = None
    X: torch.Tensor | None = None
    y: torch.Tensor | None = None
    prior_scale: float = 1.0
    Q: torch.Tensor | None = None   # optional orthogonal basis (Section 3.4)

    def c(self, dtype) -> L.pmcmc_target:
        self._keep = [_dev(t, dtype, n) for t, n in ((self.mean, "mean"), (self.prec, "prec"),
                                                    (self.X, "X"), (self.y, "y"), (self.Q, "Q"))]
        m, p, x, y, q = self._keep
        N = 0 if x is None else (x.shape[1] if self.kind == "schools" else x.shape[0])
        return L.pmcmc_target(TARGETS[self.kind], self.D, N, _ptr(m), _ptr(p), _ptr(x), _ptr(y),
                              float(self.prior_scale), _ptr(q))


@dataclass
class Options:
    sampler: str = "mala"
    step: float = 0.01
    leapfrog_L: int = 0
    jac: str = "diag"
    precision: str = "f32"
    atol: float = 1e-5
    rtol: float = 0.0
    max_iters: int = 0
    damping: float = 1.0
    clip: int = 0
    gate_grad: int = 1
    seed: int = 0
    chain_id: int = 0
    spin_limit: int = 0
    engine: str = "auto"   # "auto": tensor cores where a kernel exists; "simt": CUDA cores only
    seq_after: int = 0     # batched: complete chains unconverged after this many sweeps sequentially
    window: int = 0        # sliding-window Newton updates of this many steps (0: whole chain)

    def c(self) -> L.pmcmc_options:
        return L.pmcmc_options(SAMPLERS[self.sampler], float(self.step), int(self.leapfrog_L),
                               JACS[self.jac], PRECISIONS[self.precision], float(self.atol),
                               float(self.rtol), int(self.max_iters), float(self.damping),
                               int(self.clip), int(self.gate_grad), int(self.seed),
                               int(self.chain_id), int(self.spin_limit),
                               ENGINES[self.engine], int(self.seq_after), int(self.window))


def _result_dict(r: L.pmcmc_result) -> dict:
    return {"iters": r.iters, "status": STATUS_NAMES.get(r.status, r.status),
            "max_residual": r.max_residual, "accept_rate": r.accept_rate,
            "min_margin": r.min_margin, "nonfinite_resets": r.nonfinite_resets,
            "elapsed_ms": r.elapsed_ms, "sequential": r.sequential}


def pmcmc_gen_noise(seed: int, chain_id: int, T: int, D: int, precision: str = "f32",
                    device=None):
    """Counter-based noise (xi [T, D], u [T] float64) generated on the GPU."""
    ctx = pmcmc_create(device)
    dt = real_dtype(precision)
    xi = torch.empty((T, D), dtype=dt, device="cuda")
    u = torch.empty((T,), dtype=torch.float64, device="cuda")
    st = L.load().pmcmc_gen_noise(ctx, seed, chain_id, T, D, PRECISIONS[precision], _ptr(xi),
                                  _ptr(u), _stream())
    _check(ctx, st)
    return xi, u


def pmcmc_solve(target: Target, opt: Options, T: int, s0: torch.Tensor, s_init=None, xi=None,
                u=None, s_out=None):
    """Parallel Newton solve of the chain; returns (s [T, D], result dict)."""
    ctx = pmcmc_create()
    dt = real_dtype(opt.precision)
    s0 = _dev(s0, dt, "s0")
    s_init = _dev(s_init, dt, "s_init")
    xi = _dev(xi, dt, "xi")
    u = _dev(u, torch.float64, "u")
    if s_out is None:
        s_out = torch.empty((T, target.D), dtype=dt, device="cuda")
    tc, oc, res = target.c(dt), opt.c(), L.pmcmc_result()
    st = L.load().pmcmc_solve(ctx, C.byref(tc), C.byref(oc), T, _ptr(s0), _ptr(s_init), _ptr(xi),
                              _ptr(u), _ptr(s_out), C.byref(res), _stream())
    _check(ctx, st)
    return s_out, _result_dict(res)


def pmcmc_solve_async(target: Target, opt: Options, T: int, s0: torch.Tensor, s_init=None,
                      xi=None, u=None, s_out=None):
    """Enqueue the solve on the current stream without synchronising; returns (s [T, D],
    res_dev), res_dev a device tensor holding the pmcmc_result, to be read with
    result_from_device() once the stream has passed the solve.  The inputs are kept alive with
    the returned handle."""
    ctx = pmcmc_create()
    dt = real_dtype(opt.precision)
    s0 = _dev(s0, dt, "s0")
    s_init = _dev(s_init, dt, "s_init")
    xi = _dev(xi, dt, "xi")
    u = _dev(u, torch.float64, "u")
    if s_out is None:
        s_out = torch.empty((T, target.D), dtype=dt, device="cuda")
    res_dev = torch.zeros(C.sizeof(L.pmcmc_result), dtype=torch.uint8, device="cuda")
    tc, oc = target.c(dt), opt.c()
    st = L.load().pmcmc_solve_async(ctx, C.byref(tc), C.byref(oc), T, _ptr(s0), _ptr(s_init),
                                    _ptr(xi), _ptr(u), _ptr(s_out), _ptr(res_dev), _stream())
    _check(ctx, st)
    res_dev._keep = (s0, s_init, xi, u, target)
    return s_out, res_dev


def result_from_device(res_dev: torch.Tensor) -> dict:
    """The pmcmc_result written by pmcmc_solve_async (synchronises with the copy)."""
    raw = bytes(res_dev.cpu().numpy().tobytes())
    return _result_dict(L.pmcmc_result.from_buffer_copy(raw))


def pmcmc_seq_solve(target: Target, opt: Options, T: int, s0, xi, u, s_out=None, accept=None):
    """The sequential chain on the GPU; returns (s [T, D], accept [T] uint8)."""
    ctx = pmcmc_create()
    dt = real_dtype(opt.precision)
    s0, xi, u = _dev(s0, dt, "s0"), _dev(xi, dt, "xi"), _dev(u, torch.float64, "u")
    if s_out is None:
        s_out = torch.empty((T, target.D), dtype=dt, device="cuda")
    if accept is None:
        accept = torch.empty((T,), dtype=torch.uint8, device="cuda")
    tc, oc = target.c(dt), opt.c()
    st = L.load().pmcmc_seq_solve(ctx, C.byref(tc), C.byref(oc), T, _ptr(s0), _ptr(xi), _ptr(u),
                                  _ptr(s_out), _ptr(accept), _stream())
    _check(ctx, st)
    return s_out, accept


def pmcmc_linearize(target: Target, opt: Options, T: int, s0, s, xi, u, want_jac=True):
    """One evaluate-and-linearise pass; returns (f, J, accept, ell)."""
    ctx = pmcmc_create()
    dt = real_dtype(opt.precision)
    s0, s, xi = _dev(s0, dt, "s0"), _dev(s, dt, "s"), _dev(xi, dt, "xi")
    u = _dev(u, torch.float64, "u")
    D = target.D
    f = torch.empty((T, D), dtype=dt, device="cuda")
    J = None
    if want_jac:
        J = torch.empty((T, D, D) if opt.jac == "dense" else (T, D), dtype=dt, device="cuda")
    acc = torch.empty((T,), dtype=torch.uint8, device="cuda")
    ell = torch.empty((T,), dtype=torch.float64, device="cuda")
    tc, oc = target.c(dt), opt.c()
    st = L.load().pmcmc_linearize(ctx, C.byref(tc), C.byref(oc), T, _ptr(s0), _ptr(s), _ptr(xi),
                                  _ptr(u), _ptr(f), _ptr(J), _ptr(acc), _ptr(ell), _stream())
    _check(ctx, st)
    return f, J, acc, ell


def pmcmc_scan(kind: str, precision: str, a, b, s):
    """delta_t = a_t delta_{t-1} + b_t; s += delta (in place).  Returns s."""
    ctx = pmcmc_create()
    T, D = s.shape
    sd = real_dtype(precision)
    ad = torch.bfloat16 if precision == "f32_scan_bf16" else sd
    a, b = _dev(a, ad, "a"), _dev(b, ad, "b")
    if not s.is_contiguous() or s.dtype != sd or not s.is_cuda:
        raise ValueError("s must be a contiguous CUDA tensor of the precision's real type")
    st = L.load().pmcmc_scan(ctx, JACS[kind], PRECISIONS[precision], T, D, _ptr(a), _ptr(b),
                             _ptr(s), _stream())
    _check(ctx, st)
    return s


def pmcmc_adjoint(target: Target, opt: Options, T: int, s0, s, acc, xi, u, dL_ds,
                  jac_budget_bytes: int = 0, want_lambda: bool = False):
    """dL/d(step, prior_scale) at the fixed point with decisions held.

    Returns (d_step, d_prior_scale) or, with want_lambda, also lambda [T, D]."""
    ctx = pmcmc_create()
    dt = real_dtype(opt.precision)
    s0, s, xi, dL_ds = (_dev(s0, dt, "s0"), _dev(s, dt, "s"), _dev(xi, dt, "xi"),
                        _dev(dL_ds, dt, "dL_ds"))
    u = _dev(u, torch.float64, "u")
    acc = _dev(acc, torch.uint8, "acc")
    lam = torch.empty((T, target.D), dtype=dt, device="cuda") if want_lambda else None
    g = (C.c_double * 2)()
    tc, oc = target.c(dt), opt.c()
    st = L.load().pmcmc_adjoint(ctx, C.byref(tc), C.byref(oc), T, _ptr(s0), _ptr(s), _ptr(acc),
                                _ptr(xi), _ptr(u), _ptr(dL_ds), int(jac_budget_bytes), _ptr(lam),
                                g, _stream())
    _check(ctx, st)
    if want_lambda:
        return float(g[0]), float(g[1]), lam
    return float(g[0]), float(g[1])


class ChainSolve(torch.autograd.Function):
    """s = fixed point of the chain as a differentiable function of (step, prior_scale).

    Forward: pmcmc_solve, then one linearisation pass at the solution for the accept decisions.
    Backward: pmcmc_adjoint with those decisions held (the chain is piecewise smooth in the
    parameters; the gradient is that of the piece the solution lies on)."""

    @staticmethod
    def forward(ctx, step, prior_scale, target, opt, T, s0, xi, u, jac_budget_bytes):
        import dataclasses
        o = dataclasses.replace(opt, step=float(step))
        t = dataclasses.replace(target, prior_scale=float(prior_scale))
        s, res = pmcmc_solve(t, o, T, s0, xi=xi, u=u)
        _, _, acc, _ = pmcmc_linearize(t, dataclasses.replace(o, jac="zero"), T, s0, s, xi, u,
                                       want_jac=False)
        ctx.save_for_backward(s, acc)
        ctx.meta = (t, o, T, s0, xi, u, jac_budget_bytes)
        ctx.result = res
        return s

    @staticmethod
    def backward(ctx, grad_s):
        s, acc = ctx.saved_tensors
        t, o, T, s0, xi, u, budget = ctx.meta
        ge, gs = pmcmc_adjoint(t, o, T, s0, s, acc, xi, u, grad_s.contiguous(), budget)
        dev = grad_s.device
        return (torch.tensor(ge, dtype=torch.float64, device=dev),
                torch.tensor(gs, dtype=torch.float64, device=dev),
                None, None, None, None, None, None, None)


def solve_differentiable(target: Target, opt: Options, T: int, s0, xi, u, step, prior_scale,
                         jac_budget_bytes: int = 0):
    """Solve the chain with `step` and `prior_scale` as differentiable torch scalars."""
    return ChainSolve.apply(step, prior_scale, target, opt, T, s0, xi, u, jac_budget_bytes)


@dataclass
class ChainDesc:
    target: Target
    sampler: str
    step: float
    leapfrog_L: int
    T: int
    s0: torch.Tensor
    xi: torch.Tensor
    u: torch.Tensor
    s_out: torch.Tensor


def pmcmc_solve_batched(chains: list[ChainDesc], opt: Options):
    """Solve many chains together; returns a list of result dicts."""
    ctx = pmcmc_create()
    dt = real_dtype(opt.precision)
    arr = (L.pmcmc_chain_desc * len(chains))()
    keep = []
    for i, ch in enumerate(chains):
        tc = ch.target.c(dt)
        keep.append((tc, ch.target._keep))
        arr[i] = L.pmcmc_chain_desc(tc, SAMPLERS[ch.sampler], float(ch.step), int(ch.leapfrog_L),
                                    int(ch.T), _ptr(_dev(ch.s0, dt, "s0")), _ptr(_dev(ch.xi, dt, "xi")),
                                    _ptr(_dev(ch.u, torch.float64, "u")), _ptr(ch.s_out))
    res = (L.pmcmc_result * len(chains))()
    oc = opt.c()
    st = L.load().pmcmc_solve_batched(ctx, len(chains), arr, C.byref(oc), res, _stream())
    _check(ctx, st)
    return [_result_dict(r) for r in res]


def pmcmc_seq_solve_batched(chains: list[ChainDesc], precision: str = "f32"):
    """The sequential chains of a batch in one launch (one CTA per chain); writes each
    chain's s_out.  Asynchronous on the current stream."""
    ctx = pmcmc_create()
    dt = real_dtype(precision)
    arr = (L.pmcmc_chain_desc * len(chains))()
    keep = []
    for i, ch in enumerate(chains):
        tc = ch.target.c(dt)
        keep.append((tc, ch.target._keep))
        arr[i] = L.pmcmc_chain_desc(tc, SAMPLERS[ch.sampler], float(ch.step), int(ch.leapfrog_L),
                                    int(ch.T), _ptr(_dev(ch.s0, dt, "s0")), _ptr(_dev(ch.xi, dt, "xi")),
                                    _ptr(_dev(ch.u, torch.float64, "u")), _ptr(ch.s_out))
    oc = Options(precision=precision).c()
    st = L.load().pmcmc_seq_solve_batched(ctx, len(chains), arr, C.byref(oc), _stream())
    _check(ctx, st)


SCAN_PLAN_KERNELS = ("rows", "rows_const_d", "register", "staged", "pipe", "cluster", "wide")


def pmcmc_scan_plan(precision: str, T: int, D: int) -> dict:
    """The diagonal-scan kernel pmcmc_scan picks for T x D at `precision` (16-byte-aligned
    buffers), its timesteps per tile, the tiles of the launch and the tiles its look-back
    workspace holds.  Host-only: needs no GPU."""
    k, tile, tiles, mt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    st = L.load().pmcmc_scan_plan(JACS["diag"], PRECISIONS[precision], T, D, C.byref(k), C.byref(tile),
                                  C.byref(tiles), C.byref(mt))
    if st != L.PMCMC_OK:
        raise PmcmcError(st, f"pmcmc_scan_plan: T={T}, D={D}, precision {precision}")
    return {"kernel": SCAN_PLAN_KERNELS[k.value], "tile": tile.value, "tiles": tiles.value,
            "max_tiles": mt.value}


def pmcmc_profile_enable(enable: bool = True):
    """Start (and reset) or stop the context's launch counters and kernel event timers."""
    ctx = pmcmc_create()
    _check(ctx, L.load().pmcmc_profile_enable(ctx, int(enable)))


def pmcmc_profile_get() -> dict:
    ctx = pmcmc_create()
    p = L.pmcmc_profile()
    _check(ctx, L.load().pmcmc_profile_get(ctx, C.byref(p)))
    return {k: getattr(p, k) for k, _ in L.pmcmc_profile._fields_}


def pmcmc_scan_noalloc(precision: str, a, b, s):
    """The diagonal scan with static scratch and no context (for callers that cannot allocate:
    stream capture, fixed-budget hosts, plugins under another allocator).  In place on s."""
    T, D = s.shape
    sd = real_dtype(precision)
    ad = torch.bfloat16 if precision == "f32_scan_bf16" else sd
    a, b = _dev(a, ad, "a"), _dev(b, ad, "b")
    if not s.is_contiguous() or s.dtype != sd or not s.is_cuda:
        raise ValueError("s must be a contiguous CUDA tensor of the precision's real type")
    st = L.load().pmcmc_scan_noalloc(PRECISIONS[precision], T, D, _ptr(a), _ptr(b), _ptr(s),
                                     _stream())
    if st != 0:
        why = {L.PMCMC_EUNSUPPORTED: "look-back scratch beyond the static 8 MiB, or D > 256",
               L.PMCMC_EINVAL: "invalid arguments",
               L.PMCMC_ECUDA: "a CUDA call failed (symbol lookup, memset or launch)"}
        raise PmcmcError(st, "pmcmc_scan_noalloc: " + why.get(st, "failed"))
    return s
