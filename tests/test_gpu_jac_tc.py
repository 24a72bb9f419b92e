"""Dense logistic-MALA Jacobian assembled on the tensor cores (tcgen05 kind::tf32, one product
per term): H_t = X^T W_t X over the pairs i <= j as one GEMM per 128-timestep tile, the pairs
split over CTAs of up to 512 columns in MMA blocks of up to 256 (D = 22: one block, 25: two
blocks, 32: two CTAs).

Bars.  Against the CUDA-core FP32 assembly of the same linearisation (with the gate term the
evaluate pass is the CUDA-core one on both sides; with the gate held the tensor-core evaluate
pass feeds the tensor-core J, so f is held to the FP32 bar and steps within 1e-4 of a tie are
left out): a rejected step's J carries no H term and must agree
to FP32 rounding; an accepted step's J differs by eps times the tf32 error of the H entries,
which is at most 2^-10 (w truncated by the tensor core) + 2^-11 (Y rounded) relative per term,
so |dJ_ij| <= eps * 2e-3 * sum_n w_tn |X_ni X_nj| + 1e-5 (1 + |J_ij|).  Against the FP64
oracle's Jacobian: the FP32 bar of the other linearisation tests, 2e-3.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P

DEV = "cuda:0"


def _cu(x, dt=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dt, device=DEV)


def _linearize(gt, D, T, s0, s, xi, u, eps, gate, engine, damping=1.0, clip=0):
    opt = P.Options(sampler="mala", step=eps, jac="dense", precision="f32", gate_grad=gate, engine=engine,
                    damping=damping, clip=clip)
    f, J, acc, ell = P.pmcmc_linearize(gt, opt, T, _cu(s0), _cu(s), _cu(xi), _cu(u, torch.float64))
    torch.cuda.synchronize()
    return f.double().cpu().numpy(), J.double().cpu().numpy(), acc.cpu().numpy().astype(bool)


@pytest.mark.parametrize("gate", [0, 1])
@pytest.mark.parametrize("D,N,T", [(1, 40, 129), (5, 70, 300), (22, 130, 127), (25, 1000, 300),
                                   (32, 300, 257)])
def test_tc_dense_jacobian_matches_cuda_cores_and_oracle(D, N, T, gate):
    X, y, _ = W.blr_data(N, D, seed=D)
    X32 = X.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    gt = P.Target("logreg", D, X=_cu(X), y=_cu(y), prior_scale=1.0)
    ot = O.Target("logreg", D, X=X32, y=y32, sigma_p=1.0)
    rng = np.random.default_rng(N + D)
    s = (rng.standard_normal((T, D)) * 0.3).astype(np.float32).astype(np.float64)
    s0 = np.zeros(D)
    xi, u = W.noise(T, D, seed=7)
    xi = xi.astype(np.float32).astype(np.float64)
    eps = 0.02 if N < 1000 else 0.002
    f, J, acc = _linearize(gt, D, T, s0, s, xi, u, eps, gate, "auto")
    f2, J2, acc2 = _linearize(gt, D, T, s0, s, xi, u, eps, gate, "simt")
    prev = np.vstack([s0[None, :], s[:-1]])
    p = O.Problem(ot, "mala", eps, xi=xi, u=u, gate_grad=gate)
    logu = np.log(u)
    margin = np.array([abs(min(0.0, O.f(p, t + 1, prev[t])[1]) - logu[t]) for t in range(T)])
    if gate:  # the same CUDA-core evaluate pass on both sides
        assert np.array_equal(acc, acc2)
        np.testing.assert_array_equal(f, f2)
        keep = np.ones(T, dtype=bool)
    else:  # "auto" evaluates on the tensor cores (split tf32) as well: FP32 bar, near-ties aside
        keep = margin >= 1e-4
        assert np.array_equal(acc[keep], acc2[keep])
        np.testing.assert_allclose(f[keep], f2[keep], rtol=2e-5, atol=2e-5)
    J, J2, acc = J[keep], J2[keep], acc[keep]
    # tf32 bound of the H term, per entry
    z = prev[keep] @ X32.T
    sg = 1.0 / (1.0 + np.exp(-z))
    w = sg * (1.0 - sg)
    absxx = np.abs(np.einsum("ni,nj->nij", X32, X32)).reshape(N, D * D)
    bound = (eps * 2e-3 * (w @ absxx)).reshape(-1, D, D) * acc[:, None, None]
    bound += 1e-5 * (1.0 + np.abs(J2))
    err = np.abs(J - J2)
    assert (err <= bound).all(), (err.max(), np.unravel_index((err - bound).argmax(), err.shape))
    # the oracle's Jacobian at the same states, where the decision is not a near-tie
    idx = np.nonzero(keep)[0]
    checked = 0
    for m in range(0, len(idx), max(1, len(idx) // 40)):
        t = idx[m]
        fo, ello, acco = O.f(p, t + 1, prev[t])
        assert acc[m] == acco
        np.testing.assert_allclose(J[m], O.jacobian(p, t + 1, prev[t], "dense"), rtol=2e-3, atol=2e-3)
        checked += 1
    assert checked >= 1


def test_tc_dense_jacobian_damping_and_clip():
    D, N, T = 25, 300, 200
    X, y, _ = W.blr_data(N, D, seed=3)
    X32 = X.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    gt = P.Target("logreg", D, X=_cu(X), y=_cu(y), prior_scale=1.0)
    ot = O.Target("logreg", D, X=X32, y=y32, sigma_p=1.0)
    xi, u = W.noise(T, D, seed=8)
    xi = xi.astype(np.float32).astype(np.float64)
    eps = 0.005
    # linearise at the states of the chain itself, so that most steps are accepted
    ref, _, _ = O.chain(O.Problem(ot, "mala", eps, xi=xi, u=u), T, np.zeros(D))
    s = ref.astype(np.float32).astype(np.float64)
    # damping 3 puts every diagonal entry (about 0.7 accepted, 1 rejected) beyond 1, so the clip
    # binds there; off-diagonal entries (|3 eps H_ij| ~ 0.05) stay inside, with ~1e-3 of tf32
    # error at most
    f, J, acc = _linearize(gt, D, T, np.zeros(D), s, xi, u, eps, 1, "auto", damping=3.0, clip=1)
    f2, J2, acc2 = _linearize(gt, D, T, np.zeros(D), s, xi, u, eps, 1, "simt", damping=3.0, clip=1)
    assert np.array_equal(acc, acc2) and acc.sum() > T // 4
    assert np.abs(J).max() <= 1.0 and (np.abs(J2) == 1.0).any()
    np.testing.assert_allclose(J, J2, rtol=0, atol=1e-2)
    assert ((np.abs(J) == 1.0) != (np.abs(J2) == 1.0)).mean() <= 1e-3
