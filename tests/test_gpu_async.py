"""pmcmc_solve_async: the same solve as pmcmc_solve, enqueued without a host synchronisation,
its result written to device memory.  Bar: the same iterate bit for bit and the same result
fields as the synchronous call on the same inputs, and the oracle's trace."""
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


def test_async_matches_sync_and_oracle_fp64_dense():
    T = 256
    mu, prec, _ = W.gaussian_c1()
    xi, u = W.noise(T, 2, seed=0)
    ref, _, _ = O.chain(O.Problem(O.Target("gaussian", 2, mu=mu, P=prec), "mala", 0.1, xi=xi, u=u),
                        T, np.zeros(2))
    gt = P.Target("gaussian", 2, mean=cu(mu), prec=cu(prec))
    opt = P.Options(sampler="mala", step=0.1, jac="dense", precision="f64", atol=1e-10)
    s_a, rd = P.pmcmc_solve_async(gt, opt, T, cu(np.zeros(2)), xi=cu(xi), u=cu(u))
    ra = P.result_from_device(rd)
    s_s, rs = P.pmcmc_solve(gt, opt, T, cu(np.zeros(2)), xi=cu(xi), u=cu(u))
    assert ra["status"] == "OK" and ra["iters"] == rs["iters"]
    assert ra["max_residual"] == rs["max_residual"] and ra["accept_rate"] == rs["accept_rate"]
    assert torch.equal(s_a, s_s)
    np.testing.assert_allclose(s_a.cpu().numpy(), ref, rtol=1e-9, atol=1e-9)


def test_async_logreg_fp32_matches_sync():
    T, D, N = 3000, 8, 150
    X, y, _ = W.blr_data(N, D, seed=2)
    xi, u = W.noise(T, D, seed=4, dtype=np.float32)
    gt = P.Target("logreg", D, X=cu(X, torch.float32), y=cu(y, torch.float32))
    opt = P.Options(sampler="mala", step=0.01, jac="diag", precision="f32", atol=1e-6, clip=1,
                    gate_grad=0)
    args = (gt, opt, T, cu(np.zeros(D), torch.float32))
    s_a, rd = P.pmcmc_solve_async(*args, xi=cu(xi, torch.float32), u=cu(u))
    ra = P.result_from_device(rd)
    s_s, rs = P.pmcmc_solve(*args, xi=cu(xi, torch.float32), u=cu(u))
    assert ra["status"] == rs["status"] == "OK" and ra["iters"] == rs["iters"]
    assert torch.equal(s_a, s_s)


def test_async_empty_chain_and_unsupported_forms():
    mu, prec, _ = W.gaussian_c1()
    gt = P.Target("gaussian", 2, mean=cu(mu), prec=cu(prec))
    opt = P.Options(sampler="mala", step=0.1, jac="diag", precision="f64")
    _, rd = P.pmcmc_solve_async(gt, opt, 0, cu(np.zeros(2)))
    r = P.result_from_device(rd)
    assert r["status"] == "OK" and r["iters"] == 0
    xi, u = W.noise(64, 2, seed=1)
    with pytest.raises(P.PmcmcError):
        P.pmcmc_solve_async(gt, P.Options(sampler="mala", step=0.1, precision="f64", window=8), 64,
                            cu(np.zeros(2)), xi=cu(xi), u=cu(u))
