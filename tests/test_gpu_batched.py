"""Batched persistent solve of heterogeneous chains against the FP64 oracle, chain by chain.

FP32: max|s - s_oracle| <= 1e-5 (1 + |s|) up to the first near-tie decision (oracle margin
< 1e-4), as in the single-chain tests."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P


def cu(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def _chains(spec, seed=0):
    """spec: list of (sampler, target, D, T)."""
    out = []
    for i, (sampler, target, D, T) in enumerate(spec):
        rng_seed = 100 + 7 * i + seed
        if target == "gaussian":
            cov, prec, lam = W.random_spd(D, seed=rng_seed)
            mu = np.random.default_rng(rng_seed).standard_normal(D) * 0.3
            prec = prec.astype(np.float32).astype(np.float64)
            mu = mu.astype(np.float32).astype(np.float64)
            ot = O.Target("gaussian", D, mu=mu, P=prec)
            gt = P.Target("gaussian", D, mean=cu(mu), prec=cu(prec))
            lam_max = 1.0 / lam.min()
            step = 0.5 / lam_max if sampler == "mala" else 0.2 / np.sqrt(lam_max)
        elif target == "logreg":
            X, y, _ = W.blr_data(120, D, seed=rng_seed)
            X = X.astype(np.float32).astype(np.float64)
            ot = O.Target("logreg", D, X=X, y=y, sigma_p=1.0)
            gt = P.Target("logreg", D, X=cu(X), y=cu(y))
            step = 0.005 if sampler == "mala" else 0.02
        else:
            ot, gt = O.Target("banana", 2), P.Target("banana", 2)
            step = 0.05
        L = 8 if sampler == "hmc" else 0
        xi, u = W.noise(T, D, seed=rng_seed)
        xi = xi.astype(np.float32).astype(np.float64)
        ref, ell, acc = O.chain(O.Problem(ot, sampler, step, xi=xi, u=u, L=L), T, np.zeros(D))
        margin = np.abs(np.minimum(ell, 0) - np.log(u))
        s_out = torch.empty((T, D), dtype=torch.float32, device="cuda")
        desc = P.ChainDesc(gt, sampler, step, L, T, cu(np.zeros(D)), cu(xi), cu(u, torch.float64),
                           s_out)
        out.append((desc, ref, margin))
    return out


def _check(desc, ref, margin):
    s = desc.s_out.cpu().double().numpy()
    ties = np.nonzero(margin < 1e-4)[0]
    upto = ties[0] if len(ties) else len(ref)
    err = np.abs(s[:upto] - ref[:upto])
    bound = 1e-5 * (1 + np.abs(ref[:upto]))
    assert np.all(err <= bound), (np.max(err / bound), upto)


SPEC = [("mala", "gaussian", 2, 700), ("hmc", "gaussian", 2, 333), ("mala", "gaussian", 8, 1500),
        ("hmc", "gaussian", 8, 257), ("mala", "gaussian", 32, 900), ("hmc", "gaussian", 32, 150),
        ("mala", "logreg", 2, 400), ("hmc", "logreg", 2, 130), ("mala", "logreg", 8, 600),
        ("hmc", "logreg", 8, 97), ("mala", "logreg", 32, 300), ("mala", "banana", 2, 64),
        ("hmc", "banana", 2, 77)]


@pytest.mark.parametrize("precision", ["f32", "f32_scan_bf16"])
def test_batched_mixed_chains_match_oracle(precision):
    chains = _chains(SPEC)
    opt = P.Options(jac="diag", precision=precision, atol=1e-6, rtol=1e-6, clip=1)
    res = P.pmcmc_solve_batched([c[0] for c in chains], opt)
    for (desc, ref, margin), r in zip(chains, res):
        assert r["status"] == "OK", (desc.sampler, desc.target.kind, desc.target.D, r)
        assert r["iters"] <= desc.T + 1
        _check(desc, ref, margin)


def test_batched_repeat_call_replays_and_agrees():
    chains = _chains(SPEC[:6], seed=3)
    opt = P.Options(jac="diag", precision="f32", atol=1e-6, rtol=1e-6, clip=1)
    descs = [c[0] for c in chains]
    r1 = P.pmcmc_solve_batched(descs, opt)
    first = [d.s_out.clone() for d in descs]
    r2 = P.pmcmc_solve_batched(descs, opt)
    for a, d in zip(first, descs):
        assert torch.equal(a, d.s_out)
    assert [x["iters"] for x in r1] == [x["iters"] for x in r2]


def test_batched_rejects_bad_chains():
    chains = _chains(SPEC[:1])
    d = chains[0][0]
    bad = P.ChainDesc(d.target, "hmc", d.step, 0, d.T, d.s0, d.xi, d.u, d.s_out)
    with pytest.raises(P.PmcmcError, match="EINVAL"):
        P.pmcmc_solve_batched([bad], P.Options(jac="diag", precision="f32"))
    with pytest.raises(P.PmcmcError, match="EUNSUPPORTED"):
        P.pmcmc_solve_batched([d], P.Options(jac="dense", precision="f32"))


def test_batched_with_basis_matches_oracle():
    chains = _chains(SPEC, seed=11)
    descs = []
    for desc, ref, margin in chains:
        t = desc.target
        if t.kind == "gaussian":
            _, Q = np.linalg.eigh(t.prec.cpu().double().numpy())
        elif t.kind == "logreg":
            X = t.X.cpu().double().numpy()
            _, Q = np.linalg.eigh(X.T @ X)
        else:
            Q = None
        if Q is not None:
            t = P.Target(t.kind, t.D, mean=t.mean, prec=t.prec, X=t.X, y=t.y,
                         prior_scale=t.prior_scale, Q=cu(Q))
        descs.append(P.ChainDesc(t, desc.sampler, desc.step, desc.leapfrog_L, desc.T, desc.s0,
                                 desc.xi, desc.u, desc.s_out))
    opt = P.Options(jac="diag", precision="f32", atol=1e-6, rtol=1e-6, clip=1)
    res = P.pmcmc_solve_batched(descs, opt)
    for (_, ref, margin), d, r in zip(chains, descs, res):
        assert r["status"] == "OK", (d.sampler, d.target.kind, d.target.D, r)
        _check(d, ref, margin)


def test_batched_sequential_completion_matches_oracle():
    """With seq_after, chains not converged after that many Newton sweeps are recomputed by the
    sequential loop; every chain must then equal the oracle trace."""
    chains = _chains(SPEC, seed=5)
    descs = [c[0] for c in chains]
    opt = P.Options(jac="diag", precision="f32", atol=1e-6, rtol=1e-6, clip=1)
    full = P.pmcmc_solve_batched(descs, opt)
    cap = int(np.median([r["iters"] for r in full]))   # about half the chains need more sweeps
    opt.seq_after = cap
    res = P.pmcmc_solve_batched(descs, opt)
    assert any(r["sequential"] for r in res) and not all(r["sequential"] for r in res)
    for (desc, ref, margin), r, rf in zip(chains, res, full):
        assert r["status"] == "OK", (desc.sampler, desc.target.kind, desc.target.D, r)
        assert r["iters"] <= cap
        assert r["sequential"] == (rf["iters"] > cap)
        _check(desc, ref, margin)
