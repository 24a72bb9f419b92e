"""Seeded synthetic inputs for the parallel-Newton MCMC workloads.

This module is shared by the oracle tests, the GPU tests and the benchmark.  It holds no
arithmetic of the samplers, the Jacobians or the Newton solver: only data and noise
generation, so that the CPU oracle and the CUDA library receive identical inputs.

Input recipe (all seeds default to 0; draws are taken in the order listed):

* Bayesian logistic regression (Section 5.2 uses German Credit, which is not available here;
  these synthetic rows stand in with the same shape): ``X ~ N(0, 1)`` (N x D, row-major),
  ``w_true ~ N(0, I_D)``, ``y ~ Bernoulli(sigmoid(X w_true))``.
* Gaussian targets: mean and precision are given explicitly, or a random SPD covariance
  ``Q diag(lam) Q^T`` with ``Q`` from the QR factorisation of a Gaussian matrix and ``lam``
  log-uniform in [0.1, 10] (condition number <= 100).
* Sampler noise (Section 3.2 / Algorithm 2): ``xi_t ~ N(0, I_D)`` per step and
  ``u_t ~ U(0, 1)`` on the open interval, ``u = (k + 0.5) 2^-53`` with ``k`` a uniform 53-bit
  integer, so ``log u`` is always finite.
* Hierarchical Gaussian ("eight schools") Gibbs workload (Section 5.1, Appendix B.2): S = 8
  schools of N = 20 scores.  The paper matched its synthetic scores to a published table of
  school means and standard errors; that table is not reproduced here.  Instead school means
  ~ N(5, 10^2), school standard deviations ~ U(5, 20), scores = mean + sd * N(0, 1).  The Gibbs
  noise per sweep is the reparameterisation input: an Inv-chi^2(nu0 + S + 1, 1) variate
  (nu / chi^2_nu), 1 + S standard normals and S Inv-chi^2(alpha0 + N, 1) variates, with the
  paper's nu0 = alpha0 = 0.1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "blr_data", "gaussian_c1", "random_spd", "noise", "Chain", "batched_mix",
    "schools_data", "schools_init", "gibbs_noise", "C1", "C2", "C3", "C4", "GIBBS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def blr_data(N: int, D: int, seed: int = 0, dtype=np.float64):
    """Synthetic logistic-regression data ``(X, y, w_true)``; X ~ N(0,1), y ~ Bern(sigmoid(X w))."""
    rng = _rng(seed)
    X = rng.standard_normal((N, D))
    w_true = rng.standard_normal(D)
    p = 1.0 / (1.0 + np.exp(-(X @ w_true)))
    y = (rng.random(N) < p).astype(np.float64)
    return X.astype(dtype), y.astype(dtype), w_true


def gaussian_c1(dtype=np.float64):
    """The D=2 Gaussian of the FP64 dense-Newton workload: mean 0, covariance [[1,.9],[.9,1]]."""
    cov = np.array([[1.0, 0.9], [0.9, 1.0]])
    mu = np.zeros(2)
    prec = np.linalg.inv(cov)
    return mu.astype(dtype), prec.astype(dtype), cov


def random_spd(D: int, seed: int, lam_lo: float = 0.1, lam_hi: float = 10.0):
    """Random SPD covariance with eigenvalues log-uniform in [lam_lo, lam_hi].

    Returns ``(cov, prec, lam)`` in float64.
    """
    rng = _rng(seed)
    A = rng.standard_normal((D, D))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), size=D))
    cov = (Q * lam) @ Q.T
    prec = (Q / lam) @ Q.T
    cov = 0.5 * (cov + cov.T)
    prec = 0.5 * (prec + prec.T)
    return cov, prec, lam


def noise(T: int, D: int, seed: int = 0, dtype=np.float64):
    """Per-step sampler noise: ``xi`` (T x D, dtype) and ``u`` (T, float64, open (0,1))."""
    rng = _rng(seed)
    xi = rng.standard_normal((T, D))
    k = rng.integers(0, 2 ** 53, size=T, dtype=np.int64)
    u = (k.astype(np.float64) + 0.5) * 2.0 ** -53
    return xi.astype(dtype), u


# degrees of freedom of the two scaled-inverse-chi-square priors of the schools model (App. B.2)
SCHOOLS_NU0 = 0.1
SCHOOLS_ALPHA0 = 0.1


def schools_data(S: int = 8, N: int = 20, seed: int = 0, dtype=np.float64):
    """Scores of S schools x N students (row s = school s)."""
    rng = _rng(seed)
    means = rng.normal(5.0, 10.0, S)
    sds = rng.uniform(5.0, 20.0, S)
    X = means[:, None] + sds[:, None] * rng.standard_normal((S, N))
    return X.astype(dtype)


def schools_init(X):
    """A starting state from the data's moments: tau^2 = spread of the school means + 1,
    mu = their mean, theta_s = school means, sigma^2_s = within-school variances."""
    X = np.asarray(X, dtype=np.float64)
    m = X.mean(axis=1)
    return np.concatenate([[m.var(ddof=1) + 1.0, m.mean()], m, X.var(axis=1, ddof=1)])


def gibbs_noise(T: int, S: int, N: int, seed: int = 0, dtype=np.float64):
    """Per-sweep Gibbs noise, T x (2 + 2S), in the state's order (tau^2, mu, theta, sigma^2)."""
    rng = _rng(seed)
    nu_t = SCHOOLS_NU0 + S + 1
    nu_s = SCHOOLS_ALPHA0 + N
    xi = np.empty((T, 2 + 2 * S))
    xi[:, 0] = nu_t / rng.chisquare(nu_t, T)
    xi[:, 1:2 + S] = rng.standard_normal((T, 1 + S))
    xi[:, 2 + S:] = nu_s / rng.chisquare(nu_s, (T, S))
    return xi.astype(dtype)


# --------------------------------------------------------------------------------------------
# Named workloads (sizes as the benchmark configurations state them)
# --------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    sampler: str            # "mala" | "hmc" | "hmc_par_leapfrog"
    target: str             # "gaussian" | "logreg" | "banana"
    T: int
    D: int
    step: float
    L: int = 0
    N: int = 0
    tol: float = 1e-5
    rtol: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict)


# MALA, D=2 Gaussian, FP64, dense Newton, T=1024, step 0.1, tol 1e-10.
C1 = Workload("mala_gauss_d2_t1024_f64", "mala", "gaussian", T=1024, D=2, step=0.1, tol=1e-10)
# MALA on logistic regression N=1000, D=25, FP32, T=16384, step 0.01, tol 1e-5.
C2 = Workload("mala_logreg_n1000_d25_t16384", "mala", "logreg", T=16384, D=25, N=1000,
              step=0.01, tol=1e-5)
# HMC on the 2-D banana, L=16, step 0.05, T=100000, FP32.
C3 = Workload("hmc_banana_l16_t100000", "hmc", "banana", T=100000, D=2, L=16, step=0.05,
              tol=1e-5, rtol=1e-5)
# MALA on logistic regression N=5000, D=100, T=65536 (adjoint workload).  The step is not
# stated for this workload; 0.01 rejects every proposal from s0 = 0 (eps lambda_max(X^T W X)
# is about 16), so the step is set by the paper's own rule for MALA on logistic regression,
# about 80% acceptance (Appendix B.1): 5e-4 gives 82% on this synthetic data.
C4 = Workload("mala_logreg_n5000_d100_t65536", "mala", "logreg", T=65536, D=100, N=5000,
              step=5e-4, tol=1e-5)


# Reparameterised Gibbs on the schools model (Section 5.1): S = 8, N = 20, one chain of 2^17
# sweeps, FP32 (the paper ran chains up to 1M sweeps, in batches of 1 to 64).
GIBBS = Workload("gibbs_schools_s8_n20_t131072", "gibbs", "schools", T=131072, D=18, N=20,
                 step=0.0, tol=1e-5, rtol=1e-6)


@dataclass
class Chain:
    """One chain of the batched workload."""
    index: int
    sampler: str            # "mala" | "hmc"
    target: str             # "gaussian" | "logreg"
    D: int
    T: int
    step: float
    L: int
    mu: np.ndarray | None = None
    prec: np.ndarray | None = None
    X: np.ndarray | None = None
    y: np.ndarray | None = None
    noise_seed: int = 0


def batched_mix(n_chains: int = 512, seed: int = 0, T_lo: int = 1024, T_hi: int = 65536,
                dims=(2, 8, 32), N_logreg: int = 500, L_hmc: int = 8):
    """The mixed batched workload: MALA or HMC (L=8), D in {2, 8, 32}, Gaussian with a random
    SPD covariance (condition <= 100) or logistic regression (N=500), T ~ U[T_lo, T_hi].

    Step sizes (not given by the workload statement; chosen once here): MALA 0.5/lam_max(P)
    (Gaussian) and 0.005 (logistic); HMC 0.2/sqrt(lam_max(P)) (Gaussian) and 0.02 (logistic).
    """
    rng = _rng(seed)
    chains = []
    for c in range(n_chains):
        sampler = "mala" if rng.random() < 0.5 else "hmc"
        target = "gaussian" if rng.random() < 0.5 else "logreg"
        D = int(dims[rng.integers(0, len(dims))])
        T = int(rng.integers(T_lo, T_hi + 1))
        ch = Chain(index=c, sampler=sampler, target=target, D=D, T=T, step=0.0,
                   L=L_hmc if sampler == "hmc" else 0, noise_seed=1000 + c)
        if target == "gaussian":
            cov, prec, lam = random_spd(D, seed=10_000 + c)
            ch.mu = np.zeros(D)
            ch.prec = prec
            lam_max = 1.0 / lam.min()          # largest eigenvalue of the precision
            ch.step = 0.5 / lam_max if sampler == "mala" else 0.2 / np.sqrt(lam_max)
        else:
            X, y, _ = blr_data(N_logreg, D, seed=20_000 + c)
            ch.X, ch.y = X, y
            ch.step = 0.005 if sampler == "mala" else 0.02
        chains.append(ch)
    return chains
