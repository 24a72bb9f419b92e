"""FP64 CPU oracle for parallel-Newton MCMC (arXiv 2508.18413) — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``pmcmc_oracle.c`` (plain C99, double precision, sequential); this
module only marshals numpy arrays into it through ctypes.  Each function below names the
passage of the paper it follows; the C file carries the full statement.

Parity status: every function is pinned by an independent check in ``tests/test_oracle.py``
(finite differences, closed-form moments, library log-densities, published Philox vectors).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = [
    "Target", "Problem", "logp", "grad", "hess", "mala_step", "hmc_step", "leapfrog", "gibbs_sweep",
    "f", "chain", "jacobian", "deer", "mala_chain_frozen", "mala_adjoint", "philox4x32_10",
    "gen_noise", "SAMPLERS", "JACS",
]

SAMPLERS = {"mala": 0, "hmc": 1, "leapfrog": 2, "ula": 3, "gibbs": 4}
TARGETS = {"gaussian": 0, "logreg": 1, "banana": 2, "schools": 3}
JACS = {"dense": 0, "diag": 1, "block2": 2, "zero": 4}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _CTarget(C.Structure):
    _fields_ = [("kind", C.c_int), ("D", C.c_int), ("N", C.c_int),
                ("mu", _dp), ("P", _dp), ("X", _dp), ("y", _dp), ("sigma_p", C.c_double)]


class _CProblem(C.Structure):
    _fields_ = [("tgt", _CTarget), ("sampler", C.c_int), ("eps", C.c_double), ("L", C.c_int),
                ("gate_grad", C.c_int), ("damping", C.c_double), ("clip", C.c_int),
                ("xi", _dp), ("u", _dp)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        lib.o_logp.restype = C.c_double
        lib.o_state_dim.restype = C.c_int
        lib.o_deer.restype = C.c_int
        _lib = lib
    return _lib


def _arr(x, dtype=np.float64):
    if x is None:
        return None
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def _ptr(a, typ=_dp):
    if a is None:
        return C.cast(None, typ)
    return a.ctypes.data_as(typ)


@dataclass
class Target:
    """A target density: 'gaussian' (mu, P = precision), 'logreg' (X, y, sigma_p), 'banana',
    or 'schools' (the hierarchical Gaussian model of the Gibbs experiment, Appendix B.2: X holds
    the scores, S schools x N students, and D = 2 + 2 S)."""
    kind: str
    D: int
    mu: np.ndarray | None = None
    P: np.ndarray | None = None
    X: np.ndarray | None = None
    y: np.ndarray | None = None
    sigma_p: float = 1.0

    def __post_init__(self):
        self.mu = _arr(self.mu)
        self.P = _arr(self.P)
        self.X = _arr(self.X)
        self.y = _arr(self.y)
        if self.kind == "banana":
            assert self.D == 2
        rows = 0 if self.X is None else self.X.shape[0]
        if self.kind == "schools":
            assert self.X.ndim == 2 and self.D == 2 + 2 * self.X.shape[0]
            rows = self.X.shape[1]  # scores per school
        self._c = _CTarget(TARGETS[self.kind], self.D, rows,
                           _ptr(self.mu), _ptr(self.P), _ptr(self.X), _ptr(self.y),
                           float(self.sigma_p))


@dataclass
class Problem:
    """f_{1:T}: a sampler, a target, a step size and the per-step noise (xi, u)."""
    target: Target
    sampler: str
    eps: float
    xi: np.ndarray | None = None
    u: np.ndarray | None = None
    L: int = 0
    gate_grad: int = 1
    damping: float = 1.0
    clip: int = 0

    def __post_init__(self):
        self.xi = _arr(self.xi)
        self.u = _arr(self.u)
        self._c = _CProblem(self.target._c, SAMPLERS[self.sampler], float(self.eps), int(self.L),
                            int(self.gate_grad), float(self.damping), int(self.clip),
                            _ptr(self.xi), _ptr(self.u))

    @property
    def n(self) -> int:
        return 2 * self.target.D if self.sampler == "leapfrog" else self.target.D


# ---- targets (L0) ----------------------------------------------------------------------

def logp(t: Target, x) -> float:
    x = _arr(x)
    return _load().o_logp(C.byref(t._c), _ptr(x))


def grad(t: Target, x) -> np.ndarray:
    x = _arr(x)
    g = np.zeros(t.D)
    _load().o_grad(C.byref(t._c), _ptr(x), _ptr(g))
    return g


def hess(t: Target, x) -> np.ndarray:
    x = _arr(x)
    H = np.zeros((t.D, t.D))
    _load().o_hess(C.byref(t._c), _ptr(x), _ptr(H))
    return H


# ---- transitions (L1) ------------------------------------------------------------------

def mala_step(t: Target, eps, x, xi, u, mh=True):
    """MALA transition of Section 3.2. Returns (x_next, ell, accepted)."""
    x, xi = _arr(x), _arr(xi)
    out = np.zeros(t.D)
    ell = C.c_double()
    acc = C.c_int()
    _load().o_mala_step(C.byref(t._c), C.c_double(eps), _ptr(x), _ptr(xi), C.c_double(u),
                        C.c_int(int(mh)), _ptr(out), C.byref(ell), C.byref(acc))
    return out, ell.value, bool(acc.value)


def hmc_step(t: Target, eps, L, x, xi, u):
    """HMC transition of Algorithm 2 (sequential leapfrog). Returns (x_next, H0-HL, accepted)."""
    x, xi = _arr(x), _arr(xi)
    out = np.zeros(t.D)
    dH = C.c_double()
    acc = C.c_int()
    _load().o_hmc_step(C.byref(t._c), C.c_double(eps), C.c_int(L), _ptr(x), _ptr(xi),
                       C.c_double(u), _ptr(out), C.byref(dH), C.byref(acc))
    return out, dH.value, bool(acc.value)


def leapfrog(t: Target, eps, s):
    """One leapfrog step on s = [x, v] (Eq. 7)."""
    s = _arr(s)
    out = np.zeros(2 * t.D)
    _load().o_leapfrog(C.byref(t._c), C.c_double(eps), _ptr(s), _ptr(out))
    return out


def gibbs_sweep(t: Target, s_prev, xi):
    """One reparameterised Gibbs sweep of the schools model (Section 3.1, Appendix B.2).
    Returns (next state, its Jacobian d next / d s_prev)."""
    s_prev, xi = _arr(s_prev), _arr(xi)
    out = np.zeros(t.D)
    J = np.zeros((t.D, t.D))
    _load().o_gibbs_sweep(C.byref(t._c), _ptr(s_prev), _ptr(xi), _ptr(out), _ptr(J))
    return out, J


def f(p: Problem, t: int, s_prev):
    """f_t(s_prev) for step t (1-based). Returns (next, ell, accepted)."""
    s_prev = _arr(s_prev)
    out = np.zeros(p.n)
    ell = C.c_double()
    acc = C.c_int()
    _load().o_f(C.byref(p._c), C.c_int(t), _ptr(s_prev), _ptr(out), C.byref(ell), C.byref(acc))
    return out, ell.value, bool(acc.value)


def chain(p: Problem, T: int, s0):
    """The sequential chain s_t = f_t(s_{t-1}) (Section 2). Returns (s [T,n], ell [T], acc [T])."""
    s0 = _arr(s0)
    s = np.zeros((T, p.n))
    ell = np.zeros(T)
    acc = np.zeros(T, dtype=np.int32)
    _load().o_chain(C.byref(p._c), C.c_int(T), _ptr(s0), _ptr(s), _ptr(ell), _ptr(acc, _ip))
    return s, ell, acc.astype(bool)


# ---- Jacobians (L2) --------------------------------------------------------------------

def jacobian(p: Problem, t: int, s_prev, kind: str = "dense") -> np.ndarray:
    """Newton Jacobian at s_prev for step t: dense / diag / block2 / zero (Eqs. 2, 4, 8)."""
    s_prev = _arr(s_prev)
    J = np.zeros((p.n, p.n))
    _load().o_jac(C.byref(p._c), C.c_int(t), _ptr(s_prev), C.c_int(JACS[kind]), _ptr(J))
    return J


# ---- DEER (Eq. 3, Algorithm 1) ------------------------------------------------------------

def deer(p: Problem, T: int, s0, kind="dense", s_init=None, max_iters=None, atol=1e-10,
         rtol=0.0, rule="residual"):
    """CPU Newton solve. Returns (s [T,n], iters, converged, residual history)."""
    s0 = _arr(s0)
    s_init = _arr(s_init)
    if max_iters is None:
        max_iters = T
    s = np.zeros((T, p.n))
    hist = np.zeros(max_iters + 1)
    conv = C.c_int()
    it = _load().o_deer(C.byref(p._c), C.c_int(JACS[kind]), C.c_int(T), _ptr(s0), _ptr(s_init),
                        C.c_int(max_iters), C.c_double(atol), C.c_double(rtol),
                        C.c_int(0 if rule == "residual" else 1), _ptr(s), _ptr(hist),
                        C.byref(conv))
    n_eval = it + 1 if rule == "residual" else it
    return s, it, bool(conv.value), hist[:max(n_eval, 1)]


# ---- adjoint ------------------------------------------------------------------------------

def mala_chain_frozen(p: Problem, T: int, s0, acc):
    s0 = _arr(s0)
    acc = _arr(acc, np.int32)
    s = np.zeros((T, p.n))
    _load().o_mala_chain_frozen(C.byref(p._c), C.c_int(T), _ptr(s0), _ptr(acc, _ip), _ptr(s))
    return s


def mala_adjoint(p: Problem, T: int, s0, s, acc, dLds):
    """dL/d(eps, sigma_p) with decisions held, by the reverse recursion. Returns array(2)."""
    s0, s, dLds = _arr(s0), _arr(s), _arr(dLds)
    acc = _arr(acc, np.int32)
    g = np.zeros(2)
    _load().o_mala_adjoint(C.byref(p._c), C.c_int(T), _ptr(s0), _ptr(s), _ptr(acc, _ip),
                           _ptr(dLds), _ptr(g))
    return g


# ---- Philox and noise -----------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    _load().o_philox4x32_10(_ptr(c, u32p), _ptr(k, u32p), _ptr(out, u32p))
    return out


def gen_noise(seed: int, chain_id: int, T: int, D: int, raw: bool = False):
    """Counter-based noise: returns (xi [T,D], u [T]) and optionally the raw Philox words."""
    xi = np.zeros((T, D))
    u = np.zeros(T)
    P = (D + 1) // 2
    w = np.zeros(T * P * 4 + T * 4, dtype=np.uint32) if raw else None
    u32p = C.POINTER(C.c_uint32)
    _load().o_gen_noise(C.c_uint64(seed), C.c_uint32(chain_id), C.c_int(T), C.c_int(D),
                        _ptr(xi), _ptr(u), _ptr(w, u32p) if raw else C.cast(None, u32p))
    if raw:
        return xi, u, w
    return xi, u


def linear_recursion(A, b, dense: bool):
    """delta_t = A_t delta_{t-1} + b_t, delta_{-1} = 0 (the plain loop). Returns delta [T, n]."""
    A, b = _arr(A), _arr(b)
    T, n = b.shape
    out = np.zeros((T, n))
    _load().o_linear_recursion(C.c_int(T), C.c_int(n), C.c_int(int(dense)), _ptr(A), _ptr(b),
                               _ptr(out))
    return out


# ---- stochastic diagonal (Section 3.4, Eq. 9) -------------------------------------------------

def hutchinson_probe(seed: int, chain_id: int, t: int, it: int, D: int) -> np.ndarray:
    """Rademacher probe z (D values in {-1, +1}) of step t (0-based) at Newton iteration `it`.

    The library's counter convention: coordinate d takes bit d mod 32 of output word
    (d mod 128) div 32 of Philox4x32-10 at counter (d div 128, t, chain_id, 2 + it) under the
    key (low, high 32 bits of seed); a set bit is +1, a clear bit -1.  Philox itself is the
    known-answer-pinned generator of this module."""
    z = np.empty(D)
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    words = {}
    for d in range(D):
        blk = d >> 7
        if blk not in words:
            words[blk] = philox4x32_10([blk, t & 0xFFFFFFFF, chain_id & 0xFFFFFFFF,
                                        (2 + it) & 0xFFFFFFFF], key)
        w = int(words[blk][(d & 127) >> 5])
        z[d] = 1.0 if (w >> (d & 31)) & 1 else -1.0
    return z


def hutchinson_diag(p: Problem, t: int, s_prev, z) -> np.ndarray:
    """One-sample stochastic estimate of diag(J_t) (Eq. 9): z (.) (J_t z), with J_t the dense
    Newton Jacobian of step t (1-based) at s_prev and z a probe.  Over all sign vectors z its
    mean is diag(J_t) exactly (E[z_i z_j] = [i = j])."""
    z = _arr(z)
    return z * (jacobian(p, t, s_prev, "dense") @ z)
