"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 paths agree with the oracle to rounding (1e-9 absolute on states of size O(10));
FP32 paths to max|s - s_oracle| <= 1e-5 (1 + |s|) with identical accept decisions wherever the
oracle's decision margin |min(0, ell) - log u| exceeds 1e-4 (a near-tie may flip under FP32
state rounding; both outcomes are then valid traces of the same noise).
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


def cu(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def npy(t):
    return t.detach().cpu().double().numpy()


# ------------------------------------------------------------------------------------------
# problem builders: (oracle Target, GPU Target)
# ------------------------------------------------------------------------------------------

def gauss_pair(D, seed=5, dt=torch.float64):
    if D == 2:
        mu, prec, _ = W.gaussian_c1()
    else:
        _, prec, _ = W.random_spd(D, seed=seed)
        mu = np.random.default_rng(seed).standard_normal(D) * 0.3
    return (O.Target("gaussian", D, mu=mu, P=prec),
            P.Target("gaussian", D, mean=cu(mu, dt), prec=cu(prec, dt)))


def logreg_pair(N, D, seed=0, dt=torch.float64, sp=1.0):
    X, y, _ = W.blr_data(N, D, seed=seed)
    return (O.Target("logreg", D, X=X, y=y, sigma_p=sp),
            P.Target("logreg", D, X=cu(X, dt), y=cu(y, dt), prior_scale=sp))


def banana_pair():
    return O.Target("banana", 2), P.Target("banana", 2)


def noise(T, D, seed, dt):
    xi, u = W.noise(T, D, seed=seed)
    if dt == torch.float32:
        xi = xi.astype(np.float32).astype(np.float64)   # both sides consume the same values
    return xi, u


# ------------------------------------------------------------------------------------------
# noise (counter-based generator)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("T,D", [(1, 1), (37, 3), (4096, 25)])
def test_gen_noise_matches_oracle_generator(T, D):
    xi, u = P.pmcmc_gen_noise(seed=0xDEADBEEF12345, chain_id=17, T=T, D=D, precision="f64")
    xo, uo = O.gen_noise(0xDEADBEEF12345, 17, T, D)
    np.testing.assert_array_equal(npy(u), uo)                 # integer path: bit-exact
    np.testing.assert_allclose(npy(xi), xo, rtol=0, atol=1e-13)
    xi32, u32 = P.pmcmc_gen_noise(seed=0xDEADBEEF12345, chain_id=17, T=T, D=D, precision="f32")
    np.testing.assert_allclose(npy(xi32), xo.astype(np.float32), rtol=0, atol=1e-6)
    np.testing.assert_array_equal(npy(u32), uo)


# ------------------------------------------------------------------------------------------
# one evaluate-and-linearise pass
# ------------------------------------------------------------------------------------------

def _check_linearize(ot, gt, sampler, eps, L, jac, T, seed, dt, s_scale, s_center=None,
                     gate=1, damping=1.0, clip=0):
    D = ot.D
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((T, D)) * s_scale
    if s_center is not None:
        s = s + s_center
    s0 = rng.standard_normal(D) * s_scale + (0 if s_center is None else s_center)
    if dt == torch.float32:
        s = s.astype(np.float32).astype(np.float64)
        s0 = s0.astype(np.float32).astype(np.float64)
    xi, u = noise(T, D, seed + 1, dt)
    p = O.Problem(ot, sampler, eps, xi=xi, u=u, L=L, gate_grad=gate, damping=damping, clip=clip)
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac=jac,
                    precision="f64" if dt == torch.float64 else "f32", gate_grad=gate,
                    damping=damping, clip=clip)
    f, J, acc, ell = P.pmcmc_linearize(gt, opt, T, cu(s0, dt), cu(s, dt), cu(xi, dt), cu(u))
    f, J, acc, ell = npy(f), npy(J), npy(acc).astype(bool), npy(ell)
    logu = np.log(u)
    n_checked = 0
    for t in range(T):
        prev = s0 if t == 0 else s[t - 1]
        fo, ello, acco = O.f(p, t + 1, prev)
        margin = abs(min(0.0, ello) - logu[t])
        tight = dt == torch.float64
        if not tight and margin < 1e-4:
            continue          # near-tie under FP32 rounding: either decision is valid
        n_checked += 1
        assert acc[t] == acco, (t, ello, logu[t])
        if tight:
            np.testing.assert_allclose(f[t], fo, rtol=1e-11, atol=1e-11)
            assert ell[t] == pytest.approx(ello, rel=1e-8, abs=1e-8)
        else:
            np.testing.assert_allclose(f[t], fo, rtol=2e-5, atol=2e-5)
        if jac == "diag_hutch":
            continue
        Jo = O.jacobian(p, t + 1, prev, "dense" if jac == "dense" else "diag")
        Jg = J[t] if jac == "dense" else np.diag(J[t])
        if tight:
            np.testing.assert_allclose(Jg, Jo, rtol=1e-8, atol=1e-8)
        else:
            np.testing.assert_allclose(Jg, Jo, rtol=2e-3, atol=2e-3)
    assert n_checked >= T // 2


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac,gate", [("dense", 1), ("diag", 1), ("diag", 0)])
@pytest.mark.parametrize("D", [2, 3, 8])
def test_linearize_mala_gaussian(dt, jac, gate, D):
    ot, gt = gauss_pair(D, dt=dt)
    _check_linearize(ot, gt, "mala", 0.15, 0, jac, T=300, seed=D, dt=dt, s_scale=1.0, gate=gate)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac", ["dense", "diag"])
def test_linearize_hmc_banana(dt, jac):
    ot, gt = banana_pair()
    _check_linearize(ot, gt, "hmc", 0.05, 16, jac, T=300, seed=4, dt=dt, s_scale=2.0,
                     s_center=np.array([0.0, 9.0]))


@pytest.mark.parametrize("dt", [torch.float64])
@pytest.mark.parametrize("jac", ["dense", "diag"])
def test_linearize_hmc_gaussian(dt, jac):
    ot, gt = gauss_pair(3, dt=dt)
    _check_linearize(ot, gt, "hmc", 0.2, 5, jac, T=200, seed=9, dt=dt, s_scale=1.0)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac", ["diag", "dense"])
@pytest.mark.parametrize("N,D", [(70, 4), (130, 25)])
def test_linearize_mala_logreg(dt, jac, N, D):
    ot, gt = logreg_pair(N, D, seed=1, dt=dt)
    _check_linearize(ot, gt, "mala", 0.02, 0, jac, T=97, seed=D, dt=dt, s_scale=0.3)


def test_linearize_damping_clip():
    ot, gt = banana_pair()
    _check_linearize(ot, gt, "hmc", 0.05, 16, "dense", T=64, seed=2, dt=torch.float64,
                     s_scale=3.0, s_center=np.array([0.0, 9.0]), damping=0.5, clip=1)


# ------------------------------------------------------------------------------------------
# the scan alone
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["f64", "f32", "f32_scan_bf16"])
@pytest.mark.parametrize("T,D", [(1, 1), (7, 2), (257, 3), (5003, 25), (100003, 2), (3001, 100),
                                 (64, 256)])
def test_scan_diag_matches_linear_recursion(precision, T, D):
    rng = np.random.default_rng(T + D)
    a = rng.uniform(-0.98, 0.98, (T, D))
    b = rng.standard_normal((T, D))
    s = rng.standard_normal((T, D))
    sd = torch.float64 if precision == "f64" else torch.float32
    ad = torch.bfloat16 if precision == "f32_scan_bf16" else sd
    ag, bg = cu(a, ad), cu(b, ad)
    a_used, b_used = npy(ag), npy(bg)          # what the kernel sees (rounded storage)
    sg = cu(s, sd)
    s_in = npy(sg)
    P.pmcmc_scan("diag", precision, ag, bg, sg)
    delta = O.linear_recursion(a_used, b_used, dense=False)
    tol = 1e-12 if precision == "f64" else 2e-5
    np.testing.assert_allclose(npy(sg) - s_in, delta, rtol=tol, atol=tol * 10)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("T,D", [(1, 2), (9, 2), (1000, 2), (517, 5), (2000, 25), (300, 32)])
def test_scan_dense_matches_linear_recursion(precision, T, D):
    rng = np.random.default_rng(T * D)
    A = rng.standard_normal((T, D, D)) * (0.9 / np.sqrt(D))
    b = rng.standard_normal((T, D))
    s = rng.standard_normal((T, D))
    sd = torch.float64 if precision == "f64" else torch.float32
    ag, bg, sg = cu(A, sd), cu(b, sd), cu(s, sd)
    s_in = npy(sg)
    P.pmcmc_scan("dense", precision, ag, bg, sg)
    delta = O.linear_recursion(npy(ag), npy(bg), dense=True)
    tol = 1e-11 if precision == "f64" else 5e-5
    np.testing.assert_allclose(npy(sg) - s_in, delta, rtol=tol, atol=tol * 10)


# ------------------------------------------------------------------------------------------
# full solves against the sequential oracle trace
# ------------------------------------------------------------------------------------------

def _solve_and_compare(ot, gt, sampler, eps, L, jac, T, seed, dt, atol, rtol=0.0, clip=0,
                       damping=1.0, s0=None, tol_fp32=1e-5, max_iters=0, gate=1):
    D = ot.D
    xi, u = noise(T, D, seed, dt)
    s0 = np.zeros(D) if s0 is None else s0
    p = O.Problem(ot, "hmc" if sampler == "hmc_par_leapfrog" else sampler, eps, xi=xi, u=u, L=L)
    ref, ell, acc_ref = O.chain(p, T, s0)
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac=jac,
                    precision="f64" if dt == torch.float64 else "f32", atol=atol, rtol=rtol,
                    clip=clip, damping=damping, max_iters=max_iters, gate_grad=gate)
    s, res = P.pmcmc_solve(gt, opt, T, cu(s0, dt), xi=cu(xi, dt), u=cu(u))
    s = npy(s)
    margin = np.abs(np.minimum(ell, 0.0) - np.log(u))
    return s, res, ref, acc_ref, margin


def _assert_trace(s, ref, margin, dt, tol_fp32=1e-5):
    if dt == torch.float64:
        np.testing.assert_allclose(s, ref, rtol=1e-9, atol=1e-9)
        return
    # FP32: compare up to the first near-tie decision (after a legitimately flipped tie the
    # two traces are different valid chains of the same noise)
    ties = np.nonzero(margin < 1e-4)[0]
    upto = ties[0] if len(ties) else len(ref)
    bound = tol_fp32 * (1 + np.abs(ref[:upto]))
    err = np.abs(s[:upto] - ref[:upto])
    assert np.all(err <= bound), (np.max(err / bound), upto)
    assert upto >= min(len(ref), 300)


def test_solve_c1_dense_fp64():
    """MALA, D=2 Gaussian, FP64, dense Newton, T=1024, step 0.1, tol 1e-10."""
    c = W.C1
    ot, gt = gauss_pair(2)
    s, res, ref, acc, margin = _solve_and_compare(ot, gt, "mala", c.step, 0, "dense", c.T, 0,
                                                  torch.float64, atol=c.tol)
    assert res["status"] == "OK" and res["iters"] <= c.T
    _assert_trace(s, ref, margin, torch.float64)
    assert res["accept_rate"] == pytest.approx(acc.mean(), abs=1e-12)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac", ["diag", "dense", "zero", "diag_hutch"])
def test_solve_mala_gaussian(dt, jac):
    ot, gt = gauss_pair(3, dt=dt)
    T = 700
    atol = 1e-11 if dt == torch.float64 else 1e-6
    s, res, ref, acc, margin = _solve_and_compare(ot, gt, "mala", 0.3, 0, jac, T, 11, dt, atol=atol)
    assert res["status"] == "OK" and res["iters"] <= T
    _assert_trace(s, ref, margin, dt)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac,clip", [("diag", 1), ("dense", 0)])
def test_solve_hmc_banana(dt, jac, clip):
    ot, gt = banana_pair()
    T = 400
    atol = 1e-10 if dt == torch.float64 else 1e-5
    s, res, ref, acc, margin = _solve_and_compare(ot, gt, "hmc", 0.05, 16, jac, T, 3, dt,
                                                  atol=atol, rtol=0.0 if dt == torch.float64 else 1e-6,
                                                  clip=clip)
    assert res["status"] == "OK" and res["iters"] <= T
    _assert_trace(s, ref, margin, dt)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("jac", ["diag", "dense"])
def test_solve_mala_logreg(dt, jac):
    ot, gt = logreg_pair(150, 6, seed=2, dt=dt)
    T = 600
    atol = 1e-10 if dt == torch.float64 else 1e-6
    s, res, ref, acc, margin = _solve_and_compare(ot, gt, "mala", 0.01, 0, jac, T, 5, dt,
                                                  atol=atol, clip=1)
    assert res["status"] == "OK" and res["iters"] <= T
    _assert_trace(s, ref, margin, dt)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_solve_par_leapfrog_banana(dt):
    """Sequential HMC steps with each L=16 leapfrog recursion solved by block quasi-DEER."""
    ot, gt = banana_pair()
    T = 300
    atol = 1e-12 if dt == torch.float64 else 1e-6
    s, res, ref, acc, margin = _solve_and_compare(ot, gt, "hmc_par_leapfrog", 0.05, 16, "block2",
                                                  T, 8, dt, atol=atol, s0=np.array([0.5, 9.0]))
    assert res["status"] == "OK"
    assert res["iters"] <= T * 16
    _assert_trace(s, ref, margin, dt, tol_fp32=1e-4)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_solve_par_leapfrog_gaussian(dt):
    ot, gt = gauss_pair(3, dt=dt)
    T = 200
    atol = 1e-12 if dt == torch.float64 else 1e-6
    s, res, ref, acc, margin = _solve_and_compare(ot, gt, "hmc_par_leapfrog", 0.2, 8, "block2",
                                                  T, 4, dt, atol=atol)
    assert res["status"] == "OK"
    _assert_trace(s, ref, margin, dt, tol_fp32=1e-4)


@pytest.mark.parametrize("kind", ["mala_gauss", "hmc_banana", "mala_logreg"])
def test_seq_solve_matches_oracle(kind):
    T = 500
    if kind == "mala_gauss":
        ot, gt = gauss_pair(3)
        sampler, eps, L = "mala", 0.3, 0
    elif kind == "hmc_banana":
        ot, gt = banana_pair()
        sampler, eps, L = "hmc", 0.05, 16
    else:
        ot, gt = logreg_pair(120, 5, seed=3)
        sampler, eps, L = "mala", 0.01, 0
    xi, u = W.noise(T, ot.D, seed=21)
    ref, _, acc = O.chain(O.Problem(ot, sampler, eps, xi=xi, u=u, L=L), T, np.zeros(ot.D))
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, precision="f64")
    s, a = P.pmcmc_seq_solve(gt, opt, T, cu(np.zeros(ot.D)), cu(xi), cu(u))
    np.testing.assert_allclose(npy(s), ref, rtol=1e-10, atol=1e-10)
    np.testing.assert_array_equal(npy(a).astype(bool), acc)


@pytest.mark.parametrize("kind,jac", [("mala_gauss", "dense"), ("mala_gauss", "diag"),
                                      ("hmc_banana", "diag"), ("mala_logreg", "diag"),
                                      ("mala_logreg", "dense")])
def test_each_newton_iterate_matches_oracle_deer(kind, jac):
    """After k Newton updates from s^(0) = s0 the GPU iterate equals the oracle's DEER iterate
    (Eq. 3 form) to rounding: checks the linearisation and the scan together, per iteration."""
    T = 150
    if kind == "mala_gauss":
        ot, gt = gauss_pair(3)
        sampler, eps, L = "mala", 0.3, 0
    elif kind == "hmc_banana":
        ot, gt = banana_pair()
        sampler, eps, L = "hmc", 0.05, 16
    else:
        ot, gt = logreg_pair(90, 4, seed=7)
        sampler, eps, L = "mala", 0.01, 0
    xi, u = W.noise(T, ot.D, seed=33)
    p = O.Problem(ot, sampler, eps, xi=xi, u=u, L=L, clip=1)
    for k in (1, 2, 3, 5):
        so, it, _, _ = O.deer(p, T, np.zeros(ot.D), kind=jac, max_iters=k, atol=-1.0)
        opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac=jac, precision="f64",
                        atol=-1.0, max_iters=k, clip=1)
        s, res = P.pmcmc_solve(gt, opt, T, cu(np.zeros(ot.D)), xi=cu(xi), u=cu(u))
        assert res["iters"] == k and res["status"] == "NOT_CONVERGED"
        np.testing.assert_allclose(npy(s), so, rtol=1e-8, atol=1e-8)


def test_solve_generates_noise_from_seed():
    """xi/u omitted: the solve draws them from (seed, chain) exactly as gen_noise does."""
    ot, gt = gauss_pair(2)
    T = 300
    xo, uo = O.gen_noise(7, 3, T, 2)
    ref, _, _ = O.chain(O.Problem(ot, "mala", 0.1, xi=xo, u=uo), T, np.zeros(2))
    opt = P.Options(sampler="mala", step=0.1, jac="dense", precision="f64", atol=1e-11, seed=7,
                    chain_id=3)
    s, res = P.pmcmc_solve(gt, opt, T, cu(np.zeros(2)))
    assert res["status"] == "OK"
    np.testing.assert_allclose(npy(s), ref, rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------------------------------------
# edge cases and failure handling
# ------------------------------------------------------------------------------------------

def test_single_step_and_empty_chain():
    ot, gt = gauss_pair(2)
    xi, u = W.noise(1, 2, seed=1)
    ref, _, _ = O.chain(O.Problem(ot, "mala", 0.1, xi=xi, u=u), 1, np.ones(2))
    opt = P.Options(sampler="mala", step=0.1, jac="diag", precision="f64", atol=1e-12)
    s, res = P.pmcmc_solve(gt, opt, 1, cu(np.ones(2)), xi=cu(xi), u=cu(u))
    assert res["iters"] == 1
    np.testing.assert_allclose(npy(s), ref, rtol=1e-14)
    s, res = P.pmcmc_solve(gt, opt, 0, cu(np.ones(2)), xi=cu(np.zeros((0, 2))), u=cu(np.zeros(0)))
    assert res["status"] == "OK" and s.shape == (0, 2)


def test_invalid_arguments_are_rejected():
    ot, gt = gauss_pair(2)
    opt = P.Options(sampler="mala", step=0.1, precision="f64")
    with pytest.raises(P.PmcmcError, match="ENAN"):
        P.pmcmc_solve(gt, opt, 10, cu([np.nan, 0.0]))
    with pytest.raises(P.PmcmcError, match="EINVAL"):
        P.pmcmc_solve(gt, P.Options(sampler="mala", step=-1.0, precision="f64"), 10, cu([0.0, 0.0]))
    with pytest.raises(P.PmcmcError, match="EUNSUPPORTED"):
        X = torch.zeros((10, 200), dtype=torch.float32, device=DEV)
        y = torch.zeros(10, dtype=torch.float32, device=DEV)
        P.pmcmc_solve(P.Target("logreg", 200, X=X, y=y), P.Options(), 10,
                      torch.zeros(200, device=DEV))
    with pytest.raises(P.PmcmcError, match="EINVAL"):
        P.pmcmc_solve(gt, P.Options(sampler="mala", step=0.1, jac="block2", precision="f64"), 10,
                      cu([0.0, 0.0]))


def test_lookback_wait_bound_returns_timeout_and_context_recovers():
    """A look-back wait bound of one poll makes waits run out; the solve reports ETIMEOUT (or
    OK when no CTA had to wait) and never hangs; the context stays usable."""
    ot, gt = gauss_pair(2)
    T = 300_000
    xi, u = W.noise(T, 2, seed=2)
    xg, ug = cu(xi), cu(u)
    seen_timeout = False
    for _ in range(3):
        opt = P.Options(sampler="mala", step=0.1, jac="diag", precision="f64", atol=1e-9,
                        spin_limit=1, max_iters=3)
        try:
            P.pmcmc_solve(gt, opt, T, cu(np.zeros(2)), xi=xg, u=ug)
        except P.PmcmcError as e:
            assert e.status == -4
            seen_timeout = True
    assert seen_timeout
    # the context still solves correctly
    T2 = 500
    ref, _, _ = O.chain(O.Problem(ot, "mala", 0.1, xi=xi[:T2], u=u[:T2]), T2, np.zeros(2))
    opt = P.Options(sampler="mala", step=0.1, jac="dense", precision="f64", atol=1e-11)
    s, res = P.pmcmc_solve(gt, opt, T2, cu(np.zeros(2)), xi=xg[:T2].contiguous(),
                           u=ug[:T2].contiguous())
    assert res["status"] == "OK"
    np.testing.assert_allclose(npy(s), ref, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("kind", ["mala_logreg", "hmc_banana"])
def test_device_loop_and_host_loop_agree(kind):
    """The graph-resident Newton loop (conditional WHILE node) and the host-driven loop used
    while profiling run the same kernels: identical iterates and iteration counts."""
    T = 900
    if kind == "mala_logreg":
        ot, gt = logreg_pair(150, 6, seed=4, dt=torch.float32)
        sampler, eps, L, clip = "mala", 0.01, 0, 1
    else:
        ot, gt = banana_pair()
        sampler, eps, L, clip = "hmc", 0.05, 16, 1
    xi, u = noise(T, ot.D, 6, torch.float32)
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac="diag", precision="f32",
                    atol=1e-5, rtol=1e-6, clip=clip)
    s1, r1 = P.pmcmc_solve(gt, opt, T, cu(np.zeros(ot.D), torch.float32), xi=cu(xi, torch.float32),
                           u=cu(u))
    P.pmcmc_profile_enable(True)
    s2, r2 = P.pmcmc_solve(gt, opt, T, cu(np.zeros(ot.D), torch.float32), xi=cu(xi, torch.float32),
                           u=cu(u))
    prof = P.pmcmc_profile_get()
    P.pmcmc_profile_enable(False)
    assert r1["iters"] == r2["iters"] and r1["status"] == r2["status"] == "OK"
    assert torch.equal(s1, s2)
    assert prof["eval_launches"] == r2["iters"] + 1 and prof["scan_launches"] == r2["iters"]


# ------------------------------------------------------------------------------------------
# orthogonal reparameterisation (Section 3.4)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("sampler", ["mala", "hmc"])
def test_basis_reparam_gaussian_same_chain_fewer_iterations(dt, sampler):
    """With Q the eigenvectors of P the rotated chain is the same chain (noise rotated with it)
    and the diagonal Jacobian of Q^T J Q is exact for the linear part: far fewer iterations."""
    D, T = 8, 1500
    ot, gt = gauss_pair(D, seed=12, dt=dt)
    lam, Q = np.linalg.eigh(ot.P)
    eps = 0.5 / lam.max() if sampler == "mala" else 0.2 / np.sqrt(lam.max())
    L = 5 if sampler == "hmc" else 0
    xi, u = noise(T, D, 13, dt)
    ref, ell, acc = O.chain(O.Problem(ot, sampler, eps, xi=xi, u=u, L=L), T, np.zeros(D))
    margin = np.abs(np.minimum(ell, 0) - np.log(u))
    atol = 1e-11 if dt == torch.float64 else 1e-6
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac="diag", atol=atol,
                    precision="f64" if dt == torch.float64 else "f32")
    s_plain, r_plain = P.pmcmc_solve(gt, opt, T, cu(np.zeros(D), dt), xi=cu(xi, dt), u=cu(u))
    gq = P.Target("gaussian", D, mean=gt.mean, prec=gt.prec, Q=cu(Q, dt))
    s_q, r_q = P.pmcmc_solve(gq, opt, T, cu(np.zeros(D), dt), xi=cu(xi, dt), u=cu(u))
    assert r_q["status"] == "OK"
    _assert_trace(npy(s_q), ref, margin, dt)
    assert r_q["iters"] < r_plain["iters"]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_basis_reparam_logreg(dt):
    ot, gt = logreg_pair(200, 12, seed=5, dt=dt)
    _, V = np.linalg.eigh(ot.X.T @ ot.X)
    T = 800
    xi, u = noise(T, 12, 17, dt)
    ref, ell, acc = O.chain(O.Problem(ot, "mala", 0.005, xi=xi, u=u), T, np.zeros(12))
    margin = np.abs(np.minimum(ell, 0) - np.log(u))
    gq = P.Target("logreg", 12, X=gt.X, y=gt.y, prior_scale=1.0, Q=cu(V, dt))
    opt = P.Options(sampler="mala", step=0.005, jac="diag", clip=1,
                    atol=1e-10 if dt == torch.float64 else 1e-6,
                    precision="f64" if dt == torch.float64 else "f32")
    s, r = P.pmcmc_solve(gq, opt, T, cu(np.zeros(12), dt), xi=cu(xi, dt), u=cu(u))
    assert r["status"] == "OK"
    _assert_trace(npy(s), ref, margin, dt)


def test_fp64_polish_of_an_fp32_solve_reaches_the_oracle():
    """Mixed-precision use: an FP32 solve, then an FP64 solve started from it (s_init) polishes
    the trace to FP64 accuracy, with the oracle's decisions at every step, in fewer FP64
    iterations than an FP64 solve from the initial guess needs."""
    ot, gt64 = logreg_pair(300, 8, seed=4)
    X, y, _ = W.blr_data(300, 8, seed=4)
    gt32 = P.Target("logreg", 8, X=cu(X, torch.float32), y=cu(y, torch.float32))
    T = 3000
    xi, u = noise(T, 8, 9, torch.float32)
    ref, ell, acc = O.chain(O.Problem(ot, "mala", 0.01, xi=xi, u=u), T, np.zeros(8))
    s32, r32 = P.pmcmc_solve(gt32, P.Options(sampler="mala", step=0.01, jac="diag", precision="f32",
                                             atol=1e-6, clip=1, gate_grad=0),
                             T, cu(np.zeros(8), torch.float32), xi=cu(xi, torch.float32), u=cu(u))
    assert r32["status"] == "OK"
    o64 = P.Options(sampler="mala", step=0.01, jac="diag", precision="f64", atol=1e-11, clip=1,
                    gate_grad=0)
    s64, r64 = P.pmcmc_solve(gt64, o64, T, cu(np.zeros(8)), s_init=s32.double(), xi=cu(xi), u=cu(u))
    _, rs = P.pmcmc_solve(gt64, o64, T, cu(np.zeros(8)), xi=cu(xi), u=cu(u))
    assert r64["status"] == "OK" and rs["status"] == "OK"
    assert r64["iters"] < rs["iters"]
    np.testing.assert_allclose(npy(s64), ref, rtol=0, atol=1e-9)
    _, _, a64, _ = P.pmcmc_linearize(gt64, P.Options(sampler="mala", step=0.01, jac="zero",
                                                     precision="f64"), T, cu(np.zeros(8)), s64,
                                     cu(xi), cu(u), want_jac=False)
    np.testing.assert_array_equal(npy(a64).astype(bool), acc)
