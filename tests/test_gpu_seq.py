"""The sequential GPU loops (the baseline of every speed-up) against the FP64 oracle's chain.

The single-chain kernel keeps the logistic design in shared memory, split over a cluster of
CTAs when it does not fit one SM (PMCMC_SEQ_CLUSTER forces a cluster size here, so the
distributed-shared-memory sums run on small problems too); the many-chain kernel runs one CTA
per chain.  FP64: trace within 1e-10 and identical decisions; FP32: decisions equal wherever
the oracle's margin exceeds 1e-4 and the trace within 1e-5 (1 + |s|) up to the first such
near-tie (FP32 rounding of the states may flip a near-tie, after which both chains are valid).
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P


def cu(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def _pair(kind, D, N=0, seed=3, sp=1.0):
    if kind == "logreg":
        X, y, _ = W.blr_data(N, D, seed=seed)
        return (O.Target("logreg", D, X=X, y=y, sigma_p=sp),
                lambda dt: P.Target("logreg", D, X=cu(X, dt), y=cu(y, dt), prior_scale=sp))
    _, prec, _ = W.random_spd(D, seed=seed)
    mu = np.random.default_rng(seed).standard_normal(D) * 0.5
    return (O.Target("gaussian", D, mu=mu, P=prec),
            lambda dt: P.Target("gaussian", D, mean=cu(mu, dt), prec=cu(prec, dt)))


def _compare(s, acc_g, ref, ell, acc, u, dt):
    if dt == torch.float64:
        np.testing.assert_allclose(s, ref, rtol=1e-10, atol=1e-10)
        np.testing.assert_array_equal(acc_g, acc)
        return
    margin = np.abs(np.minimum(ell, 0.0) - np.log(u))
    near = np.nonzero(margin < 1e-4)[0]
    upto = near[0] if len(near) else len(s)
    np.testing.assert_array_equal(acc_g[:upto], acc[:upto])
    err = np.abs(s[:upto] - ref[:upto]) / (1 + np.abs(ref[:upto]))
    assert err.max() <= 1e-5, err.max()
    assert upto > 100


@pytest.mark.parametrize("cluster", ["1", "2", "4", "16"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("sampler,L", [("mala", 0), ("hmc", 3)])
def test_seq_logreg_cluster_matches_oracle(cluster, prec, sampler, L):
    dt = torch.float64 if prec == "f64" else torch.float32
    D, N, T = 7, 203, 600
    ot, gt = _pair("logreg", D, N, sp=1.3)
    eps = 0.02 if sampler == "mala" else 0.05
    xi, u = W.noise(T, D, seed=5)
    if dt == torch.float32:
        xi = xi.astype(np.float32).astype(np.float64)
    ref, ell, acc = O.chain(O.Problem(ot, sampler, eps, xi=xi, u=u, L=L), T, np.zeros(D))
    old = os.environ.get("PMCMC_SEQ_CLUSTER")
    os.environ["PMCMC_SEQ_CLUSTER"] = cluster
    try:
        s, a = P.pmcmc_seq_solve(gt(dt), P.Options(sampler=sampler, step=eps, leapfrog_L=L,
                                                   precision=prec),
                                 T, cu(np.zeros(D), dt), cu(xi, dt), cu(u))
        torch.cuda.synchronize()
    finally:
        if old is None:
            os.environ.pop("PMCMC_SEQ_CLUSTER")
        else:
            os.environ["PMCMC_SEQ_CLUSTER"] = old
    _compare(s.cpu().double().numpy(), a.cpu().numpy().astype(bool), ref, ell, acc, u, dt)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_seq_logreg_wide_state_matches_oracle(prec):
    """D = 100 (the adjoint workload's width) on a design split over a 16-CTA cluster."""
    dt = torch.float64 if prec == "f64" else torch.float32
    D, N, T = 100, 700, 300
    ot, gt = _pair("logreg", D, N, seed=8)
    xi, u = W.noise(T, D, seed=2)
    if dt == torch.float32:
        xi = xi.astype(np.float32).astype(np.float64)
    ref, ell, acc = O.chain(O.Problem(ot, "mala", 5e-4, xi=xi, u=u), T, np.zeros(D))
    os.environ["PMCMC_SEQ_CLUSTER"] = "16"
    try:
        s, a = P.pmcmc_seq_solve(gt(dt), P.Options(sampler="mala", step=5e-4, precision=prec),
                                 T, cu(np.zeros(D), dt), cu(xi, dt), cu(u))
        torch.cuda.synchronize()
    finally:
        os.environ.pop("PMCMC_SEQ_CLUSTER")
    _compare(s.cpu().double().numpy(), a.cpu().numpy().astype(bool), ref, ell, acc, u, dt)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_seq_gaussian_matches_oracle(prec):
    dt = torch.float64 if prec == "f64" else torch.float32
    for sampler, L, D in [("mala", 0, 9), ("hmc", 4, 32)]:
        ot, gt = _pair("gaussian", D, seed=D)
        T = 500
        xi, u = W.noise(T, D, seed=D + 1)
        if dt == torch.float32:
            xi = xi.astype(np.float32).astype(np.float64)
        eps = 0.1
        ref, ell, acc = O.chain(O.Problem(ot, sampler, eps, xi=xi, u=u, L=L), T, np.zeros(D))
        s, a = P.pmcmc_seq_solve(gt(dt), P.Options(sampler=sampler, step=eps, leapfrog_L=L,
                                                   precision=prec),
                                 T, cu(np.zeros(D), dt), cu(xi, dt), cu(u))
        torch.cuda.synchronize()
        _compare(s.cpu().double().numpy(), a.cpu().numpy().astype(bool), ref, ell, acc, u, dt)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_seq_batched_matches_oracle(prec):
    """Mixed chains (samplers, targets, D, T) in one launch; each against its own oracle chain."""
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(0)
    specs = []
    for i in range(11):
        kind = "logreg" if i % 2 else "gaussian"
        D = [2, 8, 32, 5][i % 4]
        sampler = "hmc" if i % 3 == 0 else "mala"
        T = int(rng.integers(50, 700))
        specs.append((kind, D, sampler, T, i))
    chains, refs = [], []
    for kind, D, sampler, T, i in specs:
        ot, gt = _pair(kind, D, N=150, seed=10 + i)
        L = 4 if sampler == "hmc" else 0
        eps = (0.01 if sampler == "mala" else 0.03) if kind == "logreg" else 0.1
        xi, u = W.noise(T, D, seed=20 + i)
        if dt == torch.float32:
            xi = xi.astype(np.float32).astype(np.float64)
        refs.append(O.chain(O.Problem(ot, sampler, eps, xi=xi, u=u, L=L), T, np.zeros(D)) + (u,))
        chains.append(P.ChainDesc(gt(dt), sampler, eps, L, T, cu(np.zeros(D), dt), cu(xi, dt),
                                  cu(u), torch.empty((T, D), dtype=dt, device="cuda")))
    P.pmcmc_seq_solve_batched(chains, precision=prec)
    torch.cuda.synchronize()
    for ch, (ref, ell, acc, u) in zip(chains, refs):
        s = ch.s_out.cpu().double().numpy()
        if dt == torch.float64:
            np.testing.assert_allclose(s, ref, rtol=1e-10, atol=1e-10)
        else:
            margin = np.abs(np.minimum(ell, 0.0) - np.log(u))
            near = np.nonzero(margin < 1e-4)[0]
            upto = near[0] if len(near) else len(s)
            err = np.abs(s[:upto] - ref[:upto]) / (1 + np.abs(ref[:upto]))
            assert err.max() <= 1e-5
