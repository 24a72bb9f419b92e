"""GPU adjoint (reverse dense scan with decisions held) against the FP64 oracle.

The oracle's reverse loop is itself pinned to central finite differences of the frozen-decision
chain (tests/test_oracle.py).  Tolerances: FP64 1e-9 relative; FP32 1e-4 relative (the reverse
recursion accumulates FP32 rounding over T steps of D x D products)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P

DEV = "cuda:0"


def cu(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def _setup(kind, T, D, N=60, eps=0.02, seed=3, sp=1.3, dt=torch.float64):
    if kind == "logreg":
        X, y, _ = W.blr_data(N, D, seed=seed)
        if dt == torch.float32:
            X = X.astype(np.float32).astype(np.float64)
        ot = O.Target("logreg", D, X=X, y=y, sigma_p=sp)
        gt = P.Target("logreg", D, X=cu(X, dt), y=cu(y, dt), prior_scale=sp)
    else:
        _, prec, _ = W.random_spd(D, seed=seed)
        mu = np.random.default_rng(seed).standard_normal(D) * 0.2
        if dt == torch.float32:
            prec = prec.astype(np.float32).astype(np.float64)
            mu = mu.astype(np.float32).astype(np.float64)
        ot = O.Target("gaussian", D, mu=mu, P=prec)
        gt = P.Target("gaussian", D, mean=cu(mu, dt), prec=cu(prec, dt))
    xi, u = W.noise(T, D, seed=seed + 1)
    if dt == torch.float32:
        xi = xi.astype(np.float32).astype(np.float64)
    p = O.Problem(ot, "mala", eps, xi=xi, u=u)
    s0 = np.zeros(D)
    s, _, acc = O.chain(p, T, s0)
    if dt == torch.float32:
        s = s.astype(np.float32).astype(np.float64)
    dLds = 2.0 * s / T
    g_ref = O.mala_adjoint(p, T, s0, s, acc, dLds)
    opt = P.Options(sampler="mala", step=eps, precision="f64" if dt == torch.float64 else "f32")
    args = (gt, opt, T, cu(s0, dt), cu(s, dt), cu(acc.astype(np.uint8), torch.uint8), cu(xi, dt),
            cu(u), cu(dLds, dt))
    return args, g_ref, (p, s, acc, dLds)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,D", [("logreg", 4), ("logreg", 25), ("gaussian", 3)])
def test_adjoint_matches_oracle(dt, kind, D):
    args, g_ref, _ = _setup(kind, T=500, D=D, dt=dt)
    ge, gs = P.pmcmc_adjoint(*args)
    rtol = 1e-9 if dt == torch.float64 else 1e-4
    assert ge == pytest.approx(g_ref[0], rel=rtol, abs=rtol * 1e-3)
    if kind == "logreg":
        assert gs == pytest.approx(g_ref[1], rel=rtol, abs=rtol * 1e-3)
    else:
        assert gs == 0.0


@pytest.mark.parametrize("budget_mats", [1, 3, 17])
def test_adjoint_recompute_segments_agree(budget_mats):
    """With a J budget of a few matrices the chain is split into many segments that rebuild
    their Jacobians; the gradient is unchanged."""
    D = 6
    args, g_ref, _ = _setup("logreg", T=400, D=D)
    full = P.pmcmc_adjoint(*args)
    seg = P.pmcmc_adjoint(*args, jac_budget_bytes=budget_mats * D * D * 8)
    np.testing.assert_allclose(seg, full, rtol=1e-11, atol=1e-14)
    assert full[0] == pytest.approx(g_ref[0], rel=1e-9)


def test_adjoint_lambda_satisfies_reverse_recursion():
    """lambda_t = dL/ds_t + J_{t+1}^T lambda_{t+1} at every step (oracle Jacobian, gate held)."""
    D, T = 5, 300
    args, _, (p, s, acc, dLds) = _setup("logreg", T=T, D=D)
    _, _, lam = P.pmcmc_adjoint(*args, want_lambda=True)
    lam = lam.cpu().numpy()
    p0 = O.Problem(p.target, "mala", p.eps, xi=p.xi, u=p.u, gate_grad=0)
    for t in range(T):
        ref = dLds[t].copy()
        if t + 1 < T:
            J = O.jacobian(p0, t + 2, s[t], "dense")
            ref += J.T @ lam[t + 1]
        np.testing.assert_allclose(lam[t], ref, rtol=1e-10, atol=1e-12)


def test_autograd_function_matches_adjoint_and_finite_differences():
    D, T, N = 4, 300, 50
    X, y, _ = W.blr_data(N, D, seed=8)
    xi, u = W.noise(T, D, seed=9)
    gt = P.Target("logreg", D, X=cu(X), y=cu(y), prior_scale=1.2)
    opt = P.Options(sampler="mala", step=0.02, jac="diag", precision="f64", atol=1e-12, clip=1)
    step = torch.tensor(0.02, dtype=torch.float64, device=DEV, requires_grad=True)
    sp = torch.tensor(1.2, dtype=torch.float64, device=DEV, requires_grad=True)
    s = P.solve_differentiable(gt, opt, T, cu(np.zeros(D)), cu(xi), cu(u), step, sp)
    loss = (s ** 2).sum() / T
    ge, gs = torch.autograd.grad(loss, (step, sp))
    # frozen-decision finite differences with the oracle
    ot = O.Target("logreg", D, X=X, y=y, sigma_p=1.2)
    ref, _, acc = O.chain(O.Problem(ot, "mala", 0.02, xi=xi, u=u), T, np.zeros(D))
    np.testing.assert_allclose(s.detach().cpu().numpy(), ref, rtol=1e-9, atol=1e-9)

    def L(e, spv):
        tt = O.Target("logreg", D, X=X, y=y, sigma_p=spv)
        ss = O.mala_chain_frozen(O.Problem(tt, "mala", e, xi=xi, u=u), T, np.zeros(D), acc)
        return (ss ** 2).sum() / T

    h = 1e-5
    fd_e = (L(0.02 * (1 + h), 1.2) - L(0.02 * (1 - h), 1.2)) / (2 * 0.02 * h)
    fd_s = (L(0.02, 1.2 + h) - L(0.02, 1.2 - h)) / (2 * h)
    assert float(ge) == pytest.approx(fd_e, rel=1e-5)
    assert float(gs) == pytest.approx(fd_s, rel=1e-5)


# ------------------------------------------------------------------------------------------
# 64 < D <= 128 in FP32: the J's come from the tensor-core kernel (split-tf32 products)
# ------------------------------------------------------------------------------------------

def _wide_setup(T=500, D=100, N=700, eps=0.002):
    # step 0.002 accepts ~90% of the steps at D = 100, N = 700; 22 data-row chunks of 32 (ragged)
    return _setup("logreg", T=T, D=D, N=N, eps=eps, dt=torch.float32)


@pytest.mark.parametrize("D,N", [(100, 700), (128, 97), (65, 300)])
def test_adjoint_tensor_core_jacobians_match_oracle(D, N):
    args, g_ref, _ = _wide_setup(D=D, N=N)
    ge, gs = P.pmcmc_adjoint(*args)
    assert ge == pytest.approx(g_ref[0], rel=1e-4)
    assert gs == pytest.approx(g_ref[1], rel=1e-4)
    # the CUDA-core kernel on the same inputs
    gt, opt = args[0], args[1]
    simt = P.Options(sampler="mala", step=opt.step, precision="f32", engine="simt")
    ge2, gs2 = P.pmcmc_adjoint(gt, simt, *args[2:])
    assert ge == pytest.approx(ge2, rel=2e-5)
    assert gs == pytest.approx(gs2, rel=2e-5)


def test_adjoint_tensor_core_lambda_satisfies_reverse_recursion():
    """Every step's J from the tensor-core kernel, checked through lambda_t = dL/ds_t +
    J_{t+1}^T lambda_{t+1} with the oracle's J (FP32 products: 1e-4 relative to the terms)."""
    T, D = 300, 100
    args, _, (p, s, acc, dLds) = _wide_setup(T=T, D=D)
    _, _, lam = P.pmcmc_adjoint(*args, want_lambda=True)
    lam = lam.double().cpu().numpy()
    p0 = O.Problem(p.target, "mala", p.eps, xi=p.xi, u=p.u, gate_grad=0)
    checked = 0
    for t in range(T - 1):
        if not acc[t + 1]:
            continue
        J = O.jacobian(p0, t + 2, s[t], "dense")
        term = J.T @ lam[t + 1]
        scale = np.abs(J.T) @ np.abs(lam[t + 1]) + np.abs(dLds[t])
        assert np.all(np.abs(lam[t] - dLds[t] - term) <= 1e-4 * scale + 1e-9), t
        checked += 1
    assert checked > T // 2


@pytest.mark.parametrize("budget_mats", [1, 7])
def test_adjoint_tensor_core_segments_agree(budget_mats):
    """Segments that rebuild a few J's each (single-step and odd pair counts) give the gradient
    of the one-segment run."""
    D = 100
    args, g_ref, _ = _wide_setup(T=200, D=D, N=300)
    full = P.pmcmc_adjoint(*args)
    seg = P.pmcmc_adjoint(*args, jac_budget_bytes=budget_mats * D * D * 4)
    np.testing.assert_allclose(seg, full, rtol=1e-5)
    assert full[0] == pytest.approx(g_ref[0], rel=1e-4)
