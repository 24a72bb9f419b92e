"""The stochastic diagonal of Eq. 9 (Section 3.4) on the GPU against the oracle.

For every step t the GPU's estimate z_t (.) (J_t z_t) is compared with the oracle's dense
Newton Jacobian (pinned by finite differences) applied to the same probe z_t, which the oracle
regenerates from its own Philox (pinned by the generator's known-answer vectors).  FP64 on both
sides: the bar is 1e-12 (1 + |estimate|) per element.
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
SEED = 0x5EED_0F_AB1E
CHAIN = 3


def cu(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def _targets(kind, D):
    if kind == "gaussian":
        _, prec, _ = W.random_spd(D, seed=4)
        mu = np.random.default_rng(4).standard_normal(D) * 0.3
        return (O.Target("gaussian", D, mu=mu, P=prec),
                P.Target("gaussian", D, mean=cu(mu), prec=cu(prec)))
    if kind == "logreg":
        X, y, _ = W.blr_data(300 if D > 8 else 60, D, seed=2)
        return (O.Target("logreg", D, X=X, y=y, sigma_p=1.2),
                P.Target("logreg", D, X=cu(X), y=cu(y), prior_scale=1.2))
    return O.Target("banana", 2), P.Target("banana", 2)


@pytest.mark.parametrize("kind,D,sampler,eps,L,gate", [
    ("gaussian", 3, "mala", 0.2, 0, 1),
    ("gaussian", 7, "mala", 0.2, 0, 0),
    ("logreg", 5, "mala", 0.05, 0, 1),
    ("logreg", 25, "mala", 0.04, 0, 1),
    ("logreg", 25, "mala", 0.04, 0, 0),
    ("banana", 2, "mala", 0.1, 0, 1),
    ("banana", 2, "hmc", 0.05, 6, 1),
    ("gaussian", 4, "hmc", 0.1, 5, 0),
])
def test_hutchinson_estimate_matches_oracle(kind, D, sampler, eps, L, gate):
    ot, gt = _targets(kind, D)
    T = 257
    rng = np.random.default_rng(31)
    scale = 0.5 if kind == "logreg" else 1.0
    s = rng.standard_normal((T, D)) * scale
    s0 = rng.standard_normal(D) * scale
    if kind == "banana":
        s[:, 1] += 9.0
        s0[1] += 9.0
    xi, u = W.noise(T, D, seed=12)
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac="diag_hutch", precision="f64",
                    gate_grad=gate, seed=SEED, chain_id=CHAIN)
    _, J, acc, _ = P.pmcmc_linearize(gt, opt, T, cu(s0), cu(s), cu(xi), cu(u))
    J = J.cpu().numpy()
    acc = acc.cpu().numpy().astype(bool)
    p = O.Problem(ot, sampler, eps, xi=xi, u=u, L=L, gate_grad=gate)
    worst = 0.0
    for t in range(T):
        prev = s0 if t == 0 else s[t - 1]
        z = O.hutchinson_probe(SEED, CHAIN, t, 0, D)
        want = O.hutchinson_diag(p, t + 1, prev, z)
        _, _, acco = O.f(p, t + 1, prev)
        assert acc[t] == acco
        err = np.abs(J[t] - want) / (1.0 + np.abs(want))
        worst = max(worst, float(err.max()))
    assert worst <= 1e-12, worst
    assert 0 < acc.sum() < T or sampler == "hmc"   # both branches of the gate were exercised
