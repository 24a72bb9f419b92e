"""Reparameterised Gibbs on the hierarchical Gaussian (schools) model: the CUDA path against the
FP64 oracle (Section 3.1, Appendix B.2).

Bars: FP64 1e-9 relative to the oracle (f, J, the Newton fixed point, the sequential chain);
FP32 f within 1e-5 (1 + |f|), J within 1e-4 (1 + |J|), traces within 1e-5 (1 + |s|)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P

DEV = "cuda:0"


def _setup(S, N, T, dt, seed=0):
    X = W.schools_data(S, N, seed=seed)
    xi = W.gibbs_noise(T, S, N, seed=seed + 1)
    if dt == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
        xi = xi.astype(np.float32).astype(np.float64)
    s0 = W.schools_init(X)
    if dt == torch.float32:
        s0 = s0.astype(np.float32).astype(np.float64)
    D = 2 + 2 * S
    ot = O.Target("schools", D, X=X)
    gt = P.Target("schools", D, X=torch.tensor(X, dtype=dt, device=DEV))
    p = O.Problem(ot, "gibbs", 0.0, xi=xi, u=np.full(T, 0.5))
    return ot, gt, p, s0, xi


def _cu(x, dt):
    return torch.tensor(np.asarray(x), dtype=dt, device=DEV)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac", ["dense", "diag"])
@pytest.mark.parametrize("S,N,T", [(8, 20, 257), (3, 5, 64), (15, 7, 33)])
def test_gibbs_linearize_matches_oracle(dt, jac, S, N, T):
    ot, gt, p, s0, xi = _setup(S, N, T, dt, seed=S)
    ref, _, _ = O.chain(p, T, s0)
    # an iterate near the chain (positive variances), perturbed
    rng = np.random.default_rng(5)
    s = ref * (1 + 0.05 * rng.standard_normal(ref.shape))
    if dt == torch.float32:
        s = s.astype(np.float32).astype(np.float64)
    prec = "f64" if dt == torch.float64 else "f32"
    opt = P.Options(sampler="gibbs", jac=jac, precision=prec)
    f, J, acc, ell = P.pmcmc_linearize(gt, opt, T, _cu(s0, dt), _cu(s, dt), _cu(xi, dt),
                                       _cu(np.full(T, 0.5), torch.float64))
    f, J = f.double().cpu().numpy(), J.double().cpu().numpy()
    assert acc.cpu().numpy().all() and np.all(ell.cpu().numpy() == 0)
    ftol, jtol = (1e-11, 1e-9) if dt == torch.float64 else (1e-5, 1e-4)
    for t in range(T):
        prev = s0 if t == 0 else s[t - 1]
        fo, Jo = O.gibbs_sweep(ot, prev, xi[t])
        np.testing.assert_allclose(f[t], fo, rtol=ftol, atol=ftol)
        if jac == "diag":
            np.testing.assert_allclose(J[t], np.diag(Jo), rtol=jtol, atol=jtol)
        else:
            np.testing.assert_allclose(J[t], Jo, rtol=jtol, atol=jtol)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_gibbs_sequential_chain_matches_oracle(dt):
    S, N, T = 8, 20, 3001
    ot, gt, p, s0, xi = _setup(S, N, T, dt)
    ref, _, _ = O.chain(p, T, s0)
    prec = "f64" if dt == torch.float64 else "f32"
    s, acc = P.pmcmc_seq_solve(gt, P.Options(sampler="gibbs", precision=prec), T, _cu(s0, dt),
                               _cu(xi, dt), _cu(np.full(T, 0.5), torch.float64))
    s = s.double().cpu().numpy()
    assert acc.cpu().numpy().all()
    tol = 1e-10 if dt == torch.float64 else 1e-5
    assert np.all(np.abs(s - ref) <= tol * (1 + np.abs(ref))), np.max(np.abs(s - ref) / (1 + np.abs(ref)))


@pytest.mark.parametrize("dt,jac,T", [(torch.float64, "dense", 700), (torch.float64, "diag", 4099),
                                      (torch.float32, "diag", 20000), (torch.float32, "dense", 2048)])
def test_gibbs_newton_solve_matches_oracle_chain(dt, jac, T):
    S, N = 8, 20
    ot, gt, p, s0, xi = _setup(S, N, T, dt, seed=2)
    ref, _, _ = O.chain(p, T, s0)
    f64 = dt == torch.float64
    opt = P.Options(sampler="gibbs", jac=jac, precision="f64" if f64 else "f32",
                    atol=1e-10 if f64 else 1e-6, rtol=1e-12 if f64 else 1e-7)
    s, res = P.pmcmc_solve(gt, opt, T, _cu(s0, dt), xi=_cu(xi, dt),
                           u=_cu(np.full(T, 0.5), torch.float64))
    assert res["status"] == "OK" and res["iters"] <= T
    s = s.double().cpu().numpy()
    tol = 1e-9 if f64 else 1e-5
    err = np.abs(s - ref) / (1 + np.abs(ref))
    assert np.all(err <= tol), (np.max(err), res)


def test_gibbs_each_newton_iterate_matches_oracle_deer():
    """FP64, dense and diagonal: after k updates the GPU iterate equals the oracle's DEER iterate
    (same Jacobian, same start s_t = s_0)."""
    S, N, T = 4, 6, 40
    ot, gt, p, s0, xi = _setup(S, N, T, torch.float64, seed=7)
    for jac in ("dense", "diag"):
        for k in (1, 2, 5):
            ref, iters, _, _ = O.deer(p, T, s0, kind=jac, max_iters=k, atol=-1.0)
            opt = P.Options(sampler="gibbs", jac=jac, precision="f64", atol=-1.0, max_iters=k)
            s, res = P.pmcmc_solve(gt, opt, T, _cu(s0, torch.float64), xi=_cu(xi, torch.float64),
                                   u=_cu(np.full(T, 0.5), torch.float64))
            assert res["iters"] == k
            np.testing.assert_allclose(s.cpu().numpy(), ref, rtol=1e-9, atol=1e-9)


def test_gibbs_argument_checks():
    S, N, T = 3, 4, 10
    ot, gt, p, s0, xi = _setup(S, N, T, torch.float64)
    s0d, xid = _cu(s0, torch.float64), _cu(xi, torch.float64)
    ud = _cu(np.full(T, 0.5), torch.float64)
    with pytest.raises(P.PmcmcError):  # Gibbs needs its reparameterisation noise
        P.pmcmc_solve(gt, P.Options(sampler="gibbs", precision="f64"), T, s0d)
    with pytest.raises(P.PmcmcError):  # the schools target is sampled by Gibbs only
        P.pmcmc_solve(gt, P.Options(sampler="mala", precision="f64"), T, s0d, xi=xid, u=ud)
    with pytest.raises(P.PmcmcError):  # no Hutchinson diagonal for Gibbs
        P.pmcmc_solve(gt, P.Options(sampler="gibbs", jac="diag_hutch", precision="f64"), T, s0d, xi=xid, u=ud)
