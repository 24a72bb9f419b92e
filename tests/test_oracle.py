"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle with an independent
fact (finite differences, closed-form stationary moments, a library log-density, a published
known-answer vector, the prefix-exactness and <= T convergence properties of Newton's method).
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------

def fd_jac(fun, x, h=1e-6):
    """Central finite-difference Jacobian of fun: R^n -> R^m at x."""
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for j in range(x.size):
        hj = h * (1.0 + abs(x[j]))
        e = np.zeros_like(x)
        e[j] = hj
        cols.append((np.asarray(fun(x + e)) - np.asarray(fun(x - e))) / (2 * hj))
    return np.stack(cols, axis=-1)


def small_logreg(N=40, D=3, seed=3, sigma_p=1.3):
    X, y, _ = W.blr_data(N, D, seed=seed)
    return O.Target("logreg", D, X=X, y=y, sigma_p=sigma_p)


def gauss(D=3, seed=5):
    cov, prec, _ = W.random_spd(D, seed=seed)
    mu = np.random.default_rng(seed).standard_normal(D)
    return O.Target("gaussian", D, mu=mu, P=prec), mu, cov


def batch_means_se(x, nb=50):
    """Standard error of the mean of an autocorrelated series by batch means."""
    n = len(x) // nb * nb
    b = x[:n].reshape(nb, -1).mean(axis=1)
    return b.std(ddof=1) / np.sqrt(nb)


# ------------------------------------------------------------------------------------------
# Philox and noise
# ------------------------------------------------------------------------------------------

def test_philox_known_answers():
    path = os.path.join(HERE, "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        out = O.philox4x32_10(w[0:4], w[4:6])
        assert list(out) == w[6:10]


def test_noise_distribution():
    xi, u = O.gen_noise(seed=12345, chain_id=7, T=40000, D=3)
    assert np.all(u > 0) and np.all(u < 1)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    for d in range(3):
        assert stats.kstest(xi[:, d], "norm").pvalue > 1e-4
    # the two Box-Muller outputs of one pair are uncorrelated
    assert abs(np.corrcoef(xi[:, 0], xi[:, 1])[0, 1]) < 0.03


def test_noise_counters_are_per_chain_and_step():
    xi1, u1 = O.gen_noise(seed=1, chain_id=0, T=8, D=4)
    xi2, u2 = O.gen_noise(seed=1, chain_id=0, T=16, D=4)
    np.testing.assert_array_equal(xi1, xi2[:8])        # prefix-stable in T
    np.testing.assert_array_equal(u1, u2[:8])
    xi3, _ = O.gen_noise(seed=1, chain_id=1, T=8, D=4)
    assert not np.allclose(xi1, xi3)
    xi4, _ = O.gen_noise(seed=1, chain_id=0, T=8, D=3)
    np.testing.assert_array_equal(xi4, xi1[:, :3])     # prefix-stable in D


# ------------------------------------------------------------------------------------------
# Targets (L0)
# ------------------------------------------------------------------------------------------

def test_gaussian_logp_matches_scipy():
    t, mu, cov = gauss(D=4)
    mvn = stats.multivariate_normal(mu, cov)
    rng = np.random.default_rng(0)
    for _ in range(5):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        assert O.logp(t, a) - O.logp(t, b) == pytest.approx(mvn.logpdf(a) - mvn.logpdf(b),
                                                            rel=1e-12, abs=1e-12)


def test_logreg_logp_matches_bernoulli_likelihood():
    X, y, _ = W.blr_data(60, 4, seed=1)
    sp = 1.7
    t = O.Target("logreg", 4, X=X, y=y, sigma_p=sp)
    rng = np.random.default_rng(2)
    for _ in range(5):
        a, b = rng.standard_normal(4), rng.standard_normal(4)

        def lp(w):
            p = 1.0 / (1.0 + np.exp(-(X @ w)))
            return stats.bernoulli.logpmf(y, p).sum() + stats.norm.logpdf(w, 0, sp).sum()

        assert O.logp(t, a) - O.logp(t, b) == pytest.approx(lp(a) - lp(b), rel=1e-10, abs=1e-10)


def test_banana_closed_form_points():
    t = O.Target("banana", 2)
    # log p = -x1^2/200 - (x2 + 0.1 x1^2 - 10)^2/2 has its maximum 0 on x = (0, 10)
    assert O.logp(t, [0.0, 10.0]) == 0.0
    assert O.logp(t, [10.0, 0.0]) == pytest.approx(-0.5)        # b = 0
    assert O.logp(t, [0.0, 0.0]) == pytest.approx(-50.0)        # b = -10
    np.testing.assert_allclose(O.grad(t, [0.0, 10.0]), [0.0, 0.0], atol=0)


@pytest.mark.parametrize("kind", ["gaussian", "logreg", "banana"])
def test_gradient_and_hessian_match_finite_differences(kind):
    if kind == "gaussian":
        t = gauss(D=4)[0]
    elif kind == "logreg":
        t = small_logreg(N=80, D=4)
    else:
        t = O.Target("banana", 2)
    rng = np.random.default_rng(11)
    for _ in range(4):
        x = rng.standard_normal(t.D) * (3.0 if kind == "banana" else 0.7)
        g_fd = fd_jac(lambda z: np.array([O.logp(t, z)]), x)[0]
        np.testing.assert_allclose(O.grad(t, x), g_fd, rtol=1e-6, atol=1e-6)
        H_fd = fd_jac(lambda z: O.grad(t, z), x)
        np.testing.assert_allclose(O.hess(t, x), H_fd, rtol=1e-6, atol=1e-6)


# ------------------------------------------------------------------------------------------
# Transitions (L1)
# ------------------------------------------------------------------------------------------

def test_mala_ratio_matches_library_proposal_densities():
    """ell = log p(x~) + log q(x|x~) - log p(x) - log q(x~|x), q = N(b + eps grad(b), 2 eps I)."""
    t = small_logreg(N=50, D=3)
    eps = 0.05
    rng = np.random.default_rng(4)
    for _ in range(6):
        x, xi = rng.standard_normal(3) * 0.5, rng.standard_normal(3)
        xt = x + eps * O.grad(t, x) + np.sqrt(2 * eps) * xi
        cov = 2 * eps * np.eye(3)
        ref = (O.logp(t, xt) - O.logp(t, x)
               + stats.multivariate_normal(xt + eps * O.grad(t, xt), cov).logpdf(x)
               - stats.multivariate_normal(x + eps * O.grad(t, x), cov).logpdf(xt))
        _, ell, _ = O.mala_step(t, eps, x, xi, 0.5)
        assert ell == pytest.approx(ref, rel=1e-10, abs=1e-10)
        # the proposal is the ULA step
        np.testing.assert_allclose(O.mala_step(t, eps, x, xi, 0.5, mh=False)[0], xt, rtol=1e-14)


def test_mala_accepts_strictly_above_log_u():
    t = gauss(D=2)[0]
    x, xi = np.array([1.5, -0.7]), np.array([0.3, 2.0])
    _, ell, _ = O.mala_step(t, 0.3, x, xi, 0.5)
    assert ell < 0
    u_lo, u_hi = np.exp(ell) * (1 - 1e-9), np.exp(ell) * (1 + 1e-9)
    assert O.mala_step(t, 0.3, x, xi, u_lo)[2]
    assert not O.mala_step(t, 0.3, x, xi, u_hi)[2]
    np.testing.assert_array_equal(O.mala_step(t, 0.3, x, xi, u_hi)[0], x)


def _long_chain(sampler, target, eps, T, L=0, seed=0):
    xi, u = W.noise(T, target.D, seed=seed)
    p = O.Problem(target, sampler, eps, xi=xi, u=u, L=L)
    s, _, acc = O.chain(p, T, np.zeros(target.D))
    return s, acc


@pytest.mark.parametrize("sampler,eps,L", [("mala", 0.1, 0), ("hmc", 0.1, 10)])
def test_gaussian_chain_has_target_moments(sampler, eps, L):
    """MALA and HMC leave N(0, Sigma) invariant: the chain's mean and covariance match."""
    mu, prec, cov = W.gaussian_c1()
    t = O.Target("gaussian", 2, mu=mu, P=prec)
    s, acc = _long_chain(sampler, t, eps, 200_000, L=L, seed=7)
    s = s[2000:]
    for d in range(2):
        assert abs(s[:, d].mean()) < 5 * batch_means_se(s[:, d]) + 1e-3
        v = (s[:, d] - 0.0) ** 2
        assert abs(v.mean() - cov[d, d]) < 5 * batch_means_se(v) + 1e-3
    cxy = s[:, 0] * s[:, 1]
    assert abs(cxy.mean() - cov[0, 1]) < 5 * batch_means_se(cxy) + 1e-3


def test_ula_chain_has_closed_form_covariance():
    """Without the MH step the Gaussian chain is affine; in the eigenbasis of P its stationary
    variance is 2 eps / (1 - (1 - eps lam)^2), which differs from 1/lam (Section 2's affine
    case).  This pins the proposal and separates MALA from ULA."""
    mu, prec, cov = W.gaussian_c1()
    t = O.Target("gaussian", 2, mu=mu, P=prec)
    eps = 0.1
    s, _ = _long_chain("ula", t, eps, 200_000, seed=9)
    lam, Q = np.linalg.eigh(prec)
    z = s[2000:] @ Q
    for i in range(2):
        expected = 2 * eps / (1 - (1 - eps * lam[i]) ** 2)
        v = z[:, i] ** 2
        assert abs(v.mean() - expected) < 5 * batch_means_se(v) + 1e-3
    assert abs(2 * eps / (1 - (1 - eps * lam[1]) ** 2) - 1 / lam[1]) > 0.05


def test_banana_hmc_moments():
    """x1 ~ N(0, 100), x2 | x1 ~ N(10 - 0.1 x1^2, 1): E x2 = 0, Var x1 = 100, Var x2 = 201."""
    t = O.Target("banana", 2)
    s, acc = _long_chain("hmc", t, 0.2, 200_000, L=50, seed=2)
    s = s[5000:]
    assert acc.mean() > 0.5
    m1, m2 = s[:, 0].mean(), s[:, 1].mean()
    assert abs(m1) < 5 * batch_means_se(s[:, 0]) + 0.1
    assert abs(m2) < 5 * batch_means_se(s[:, 1]) + 0.1
    v1 = s[:, 0] ** 2
    assert abs(v1.mean() - 100) < 5 * batch_means_se(v1) + 1.0
    v2 = (s[:, 1]) ** 2
    assert abs(v2.mean() - 201) < 5 * batch_means_se(v2) + 2.0


def test_leapfrog_is_eq7():
    """Two leapfrog steps composed agree with the symplectic-Euler map of Eq. 7 applied twice,
    and its Jacobian has unit determinant (volume preservation)."""
    t = O.Target("banana", 2)
    s = np.array([1.2, 3.4, -0.3, 0.8])
    J = fd_jac(lambda z: O.leapfrog(t, 0.05, z), s)
    assert np.linalg.det(J) == pytest.approx(1.0, abs=1e-8)
    xp = s[:2] + 0.05 * s[2:]
    np.testing.assert_allclose(O.leapfrog(t, 0.05, s)[:2], xp, rtol=1e-15)


def test_leapfrog_on_a_gaussian_is_the_linear_map_of_eq7():
    """On a Gaussian target grad log p(x) = -P (x - mu) is affine, so one leapfrog step
    (x' = x + eps v, v' = v + eps grad log p(x')) is the linear map
    [[I, eps I], [-eps P, I - eps^2 P]] on (x - mu, v).  A sign or argument error in the
    velocity update (v' from grad log p at x instead of x', or v' = v - eps grad) fails it."""
    t, mu, _ = gauss(D=3, seed=11)
    P_ = t.P
    eps = 0.07
    I = np.eye(3)
    M = np.block([[I, eps * I], [-eps * P_, I - eps * eps * P_]])
    rng = np.random.default_rng(4)
    for _ in range(5):
        s = rng.standard_normal(6) * 2.0
        want = M @ np.concatenate([s[:3] - mu, s[3:]]) + np.concatenate([mu, np.zeros(3)])
        np.testing.assert_allclose(O.leapfrog(t, eps, s), want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["gaussian", "banana"])
def test_leapfrog_steps_reproduce_the_hmc_proposal(kind):
    """Algorithm 2 with the half-step bookkeeping of Appendix A.2: L leapfrog steps from
    [x_0, v_0 + (eps/2) grad log p(x_0)], then v_L - (eps/2) grad log p(x_L), give the HMC
    proposal; with u -> 0 (always accept) the moment-pinned HMC step returns that proposal, and
    its energy change H_0 - H_L follows from the final (x_L, v_L)."""
    t = gauss(D=3, seed=2)[0] if kind == "gaussian" else O.Target("banana", 2)
    eps, L = (0.1, 7) if kind == "gaussian" else (0.05, 16)
    rng = np.random.default_rng(9)
    for _ in range(4):
        x0 = rng.standard_normal(t.D) + (np.array([0.0, 9.0]) if kind == "banana" else 0.0)
        v0 = rng.standard_normal(t.D)
        s = np.concatenate([x0, v0 + 0.5 * eps * O.grad(t, x0)])
        for _k in range(L):
            s = O.leapfrog(t, eps, s)
        xL = s[:t.D]
        vL = s[t.D:] - 0.5 * eps * O.grad(t, xL)
        out, dH, acc = O.hmc_step(t, eps, L, x0, v0, 1e-300)
        assert acc
        np.testing.assert_allclose(out, xL, rtol=1e-12, atol=1e-12)
        H0 = 0.5 * v0 @ v0 - O.logp(t, x0)
        HL = 0.5 * vL @ vL - O.logp(t, xL)
        assert dH == pytest.approx(H0 - HL, rel=1e-10, abs=1e-10)


# ------------------------------------------------------------------------------------------
# Newton Jacobians (L2)
# ------------------------------------------------------------------------------------------

def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def _mala_pieces(t, eps, xi, u):
    def prop(x):
        return O.mala_step(t, eps, x, xi, u, mh=False)[0]

    def gtilde(x):
        _, ell, _ = O.mala_step(t, eps, x, xi, u)
        return min(0.0, ell) - np.log(u)

    return prop, gtilde


@pytest.mark.parametrize("kind", ["gaussian", "logreg", "banana"])
def test_mala_jacobian_is_stop_gradient_relaxation(kind):
    """J_sg = d/dx[sigma(g~) x~ + (1 - sigma(g~)) x] + (1(g~>0) - sigma(g~)) (dx~/dx - I)."""
    if kind == "gaussian":
        t = gauss(D=3)[0]
    elif kind == "logreg":
        t = small_logreg(N=40, D=3)
    else:
        t = O.Target("banana", 2)
    eps = 0.2 if kind != "logreg" else 0.3
    rng = np.random.default_rng(21)
    n_active = 0
    for trial in range(60):
        if n_active >= 4:
            break
        x = rng.standard_normal(t.D)
        if kind == "banana":        # start on the ridge x2 = 10 - 0.1 x1^2 of the target
            x = np.array([3 * x[0], 10 - 0.3 * x[0] ** 2 + x[1]])
        xi = rng.standard_normal(t.D)
        u = rng.uniform(0.05, 0.95)
        prop, gtilde = _mala_pieces(t, eps, xi, u)
        g0 = gtilde(x)
        _, ell, acc = O.mala_step(t, eps, x, xi, u)
        if abs(ell) < 1e-3 or abs(g0) < 1e-3:
            continue
        n_active += ell < 0
        relaxed = lambda z: _sig(gtilde(z)) * prop(z) + (1 - _sig(gtilde(z))) * z
        Jr = fd_jac(relaxed, x)
        Jp = fd_jac(prop, x)
        expected = Jr + (float(acc) - _sig(g0)) * (Jp - np.eye(t.D))
        p = O.Problem(t, "mala", eps, xi=xi[None, :], u=np.array([u]))
        J = O.jacobian(p, 1, x, "dense")
        np.testing.assert_allclose(J, expected, rtol=1e-5, atol=1e-6)
        # the held-gate Jacobian drops only the sigma' term
        p0 = O.Problem(t, "mala", eps, xi=xi[None, :], u=np.array([u]), gate_grad=0)
        J0 = O.jacobian(p0, 1, x, "dense")
        np.testing.assert_allclose(J0, float(acc) * Jp + (1 - float(acc)) * np.eye(t.D),
                                   rtol=1e-5, atol=1e-6)
    assert n_active >= 2


@pytest.mark.parametrize("kind", ["gaussian", "banana", "logreg"])
def test_hmc_jacobian_is_stop_gradient_relaxation(kind):
    if kind == "gaussian":
        t = gauss(D=3)[0]
        eps, L = 0.2, 5
    elif kind == "logreg":
        t = small_logreg(N=30, D=3)
        eps, L = 0.05, 4
    else:
        t = O.Target("banana", 2)
        eps, L = 0.05, 16
    rng = np.random.default_rng(8)
    n_active = 0
    for trial in range(60):
        if n_active >= 4:
            break
        x = rng.standard_normal(t.D)
        if kind == "banana":        # start on the ridge x2 = 10 - 0.1 x1^2 of the target
            x = np.array([3 * x[0], 10 - 0.3 * x[0] ** 2 + x[1]])
        xi = rng.standard_normal(t.D)
        u = rng.uniform(0.05, 0.95)

        def prop(z):
            return O.hmc_step(t, eps, L, z, xi, 1e-300)[0]

        def gtilde(z):
            return min(0.0, O.hmc_step(t, eps, L, z, xi, u)[1]) - np.log(u)

        _, dH, acc = O.hmc_step(t, eps, L, x, xi, u)
        g0 = gtilde(x)
        if abs(dH) < 1e-3 or abs(g0) < 1e-3:
            continue
        n_active += dH < 0
        relaxed = lambda z: _sig(gtilde(z)) * prop(z) + (1 - _sig(gtilde(z))) * z
        expected = fd_jac(relaxed, x) + (float(acc) - _sig(g0)) * (fd_jac(prop, x) - np.eye(t.D))
        p = O.Problem(t, "hmc", eps, xi=xi[None, :], u=np.array([u]), L=L)
        np.testing.assert_allclose(O.jacobian(p, 1, x, "dense"), expected, rtol=1e-5, atol=1e-6)
    assert n_active >= 2


def test_leapfrog_jacobian_and_block_form():
    t = small_logreg(N=30, D=3)
    p = O.Problem(t, "leapfrog", 0.07)
    s = np.random.default_rng(1).standard_normal(6)
    J = O.jacobian(p, 1, s, "dense")
    np.testing.assert_allclose(J, fd_jac(lambda z: O.leapfrog(t, 0.07, z), s), rtol=1e-6, atol=1e-7)
    Jb = O.jacobian(p, 1, s, "block2")
    # block quasi-DEER keeps exactly the diagonal of each D x D block (Appendix A.3)
    mask = np.zeros((6, 6), bool)
    for i in range(6):
        for j in range(6):
            mask[i, j] = (i % 3) == (j % 3)
    np.testing.assert_array_equal(Jb[mask], J[mask])
    assert np.all(Jb[~mask] == 0)
    Jd = O.jacobian(p, 1, s, "diag")
    np.testing.assert_array_equal(np.diag(Jd), np.diag(J))
    assert np.count_nonzero(Jd - np.diag(np.diag(Jd))) == 0


@pytest.mark.parametrize("kind,sampler", [("gaussian", "mala"), ("logreg", "mala"),
                                          ("banana", "mala"), ("banana", "hmc"),
                                          ("gaussian", "hmc")])
def test_hutchinson_estimate_is_unbiased_by_enumeration(kind, sampler):
    """Eq. 9: E_z[z (.) (J z)] = diag J for Rademacher z.  The mean over all 2^D sign vectors is
    exact, so it must equal the diagonal of the Jacobian, which the finite-difference pins above
    fix; a probe applied on the wrong side (z (.) J^T z has the same mean, so also check one z by
    hand), a dropped z factor or a transposed operand fails it."""
    import itertools
    if kind == "gaussian":
        t = gauss(D=3, seed=8)[0]
    elif kind == "logreg":
        t = small_logreg(N=30, D=4, seed=6)
    else:
        t = O.Target("banana", 2)
    D = t.D
    rng = np.random.default_rng(17)
    eps, L = (0.2, 0) if sampler == "mala" else (0.05, 5)
    for trial in range(3):
        x = rng.standard_normal(D) + (np.array([0.0, 9.0]) if kind == "banana" else 0.0)
        xi = rng.standard_normal(D)
        u = rng.uniform(0.05, 0.95)
        p = O.Problem(t, sampler, eps, xi=xi[None, :], u=np.array([u]), L=L)
        Jd = O.jacobian(p, 1, x, "dense")
        est = np.zeros(D)
        for signs in itertools.product([-1.0, 1.0], repeat=D):
            est += O.hutchinson_diag(p, 1, x, np.array(signs))
        est /= 2 ** D
        np.testing.assert_allclose(est, np.diag(Jd), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(np.diag(O.jacobian(p, 1, x, "diag")), np.diag(Jd),
                                   rtol=1e-13, atol=1e-13)
        z = np.where(rng.random(D) < 0.5, -1.0, 1.0)
        by_hand = np.array([z[i] * sum(Jd[i, j] * z[j] for j in range(D)) for i in range(D)])
        np.testing.assert_allclose(O.hutchinson_diag(p, 1, x, z), by_hand, rtol=1e-14, atol=1e-14)


def test_hutchinson_probe_is_rademacher_from_philox():
    """The probe's signs are balanced and independent across coordinates, steps and Newton
    iterations (they come from distinct Philox counters), and coordinate d >= 128 moves to the
    next counter block."""
    Z = np.array([O.hutchinson_probe(0xABCDEF0123, 3, t, 0, 40) for t in range(400)])
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 0.03
    C_ = np.corrcoef(Z.T)
    assert np.max(np.abs(C_ - np.eye(40))) < 0.25
    z0 = O.hutchinson_probe(5, 0, 7, 0, 200)
    z1 = O.hutchinson_probe(5, 0, 7, 1, 200)
    assert np.mean(z0 == z1) < 0.7              # a new probe per Newton iteration
    w = O.philox4x32_10([1, 7, 0, 2], [5, 0])   # coordinate 130 = bit 2 of word 0, block 1
    assert z0[130] == (1.0 if (int(w[0]) >> 2) & 1 else -1.0)


def test_damping_and_clip():
    t = O.Target("banana", 2)
    xi, u = np.array([[0.4, -1.0]]), np.array([0.3])
    x = np.array([4.0, -3.0])
    J = O.jacobian(O.Problem(t, "hmc", 0.05, xi=xi, u=u, L=16), 1, x, "dense")
    Jc = O.jacobian(O.Problem(t, "hmc", 0.05, xi=xi, u=u, L=16, damping=0.5, clip=1), 1, x, "dense")
    np.testing.assert_allclose(Jc, np.clip(0.5 * J, -1, 1), rtol=1e-15)


def test_block_composition_formula():
    """Appendix A.3: the product of two 2x2-block matrices with diagonal blocks has diagonal
    blocks (ae+bg, af+bh; ce+dg, cf+dh) -- 8 elementwise products."""
    rng = np.random.default_rng(0)
    D = 5
    a, b, c, d, e, f, g, h = rng.standard_normal((8, D))
    A = np.block([[np.diag(a), np.diag(b)], [np.diag(c), np.diag(d)]])
    B = np.block([[np.diag(e), np.diag(f)], [np.diag(g), np.diag(h)]])
    AB = A @ B
    np.testing.assert_allclose(np.diag(AB[:D, :D]), a * e + b * g, rtol=1e-14)
    np.testing.assert_allclose(np.diag(AB[:D, D:]), a * f + b * h, rtol=1e-14)
    np.testing.assert_allclose(np.diag(AB[D:, :D]), c * e + d * g, rtol=1e-14)
    np.testing.assert_allclose(np.diag(AB[D:, D:]), c * f + d * h, rtol=1e-14)
    off = AB.copy()
    for i in range(2 * D):
        for j in range(2 * D):
            if i % D == j % D:
                off[i, j] = 0
    assert np.abs(off).max() == 0


# ------------------------------------------------------------------------------------------
# DEER: convergence to the sequential trace, prefix exactness, <= T iterations
# ------------------------------------------------------------------------------------------

def _problem(kind, T, seed=0):
    if kind == "mala_gauss":
        mu, prec, _ = W.gaussian_c1()
        t = O.Target("gaussian", 2, mu=mu, P=prec)
        xi, u = W.noise(T, 2, seed=seed)
        return O.Problem(t, "mala", 0.1, xi=xi, u=u), np.zeros(2)
    if kind == "mala_logreg":
        t = small_logreg(N=60, D=4, sigma_p=1.0)
        xi, u = W.noise(T, 4, seed=seed)
        return O.Problem(t, "mala", 0.02, xi=xi, u=u), np.zeros(4)
    if kind == "hmc_banana":
        t = O.Target("banana", 2)
        xi, u = W.noise(T, 2, seed=seed)
        return O.Problem(t, "hmc", 0.05, xi=xi, u=u, L=16), np.zeros(2)
    if kind == "leapfrog_logreg":
        t = small_logreg(N=60, D=4, sigma_p=1.0)
        return O.Problem(t, "leapfrog", 0.05), np.random.default_rng(1).standard_normal(8)
    raise KeyError(kind)


@pytest.mark.parametrize("kind,jac", [
    ("mala_gauss", "dense"), ("mala_gauss", "diag"), ("mala_gauss", "zero"),
    ("mala_logreg", "diag"), ("mala_logreg", "dense"), ("hmc_banana", "diag"),
    ("hmc_banana", "dense"), ("leapfrog_logreg", "block2"), ("leapfrog_logreg", "diag"),
])
def test_deer_reaches_sequential_trace(kind, jac):
    T = 48
    p, s0 = _problem(kind, T)
    ref, _, _ = O.chain(p, T, s0)
    s, iters, conv, hist = O.deer(p, T, s0, kind=jac, atol=1e-11)
    assert conv
    assert iters <= T
    np.testing.assert_allclose(s, ref, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("kind,jac", [("mala_gauss", "diag"), ("hmc_banana", "diag"),
                                      ("mala_logreg", "dense"), ("leapfrog_logreg", "block2")])
def test_deer_prefix_is_exact_after_k_iterations(kind, jac):
    """After k Newton updates from any guess, s_1..s_k equal the sequential trace (Section 2:
    s_1 = f_1(s_0) is exact after one update, and induction)."""
    T = 24
    p, s0 = _problem(kind, T, seed=3)
    ref, _, _ = O.chain(p, T, s0)
    for k in range(1, 8):
        s, iters, _, _ = O.deer(p, T, s0, kind=jac, max_iters=k, atol=-1.0)
        assert iters == k
        np.testing.assert_allclose(s[:k], ref[:k], rtol=1e-11, atol=1e-11)


def test_dense_deer_solves_affine_chain_in_one_update():
    """ULA on a Gaussian is affine, so the exact-Jacobian Newton step is exact (Section 2)."""
    _, prec, _ = W.gaussian_c1()
    t = O.Target("gaussian", 2, mu=np.array([0.3, -0.2]), P=prec)
    T = 200
    xi, u = W.noise(T, 2, seed=4)
    p = O.Problem(t, "ula", 0.1, xi=xi, u=u)
    s, iters, conv, hist = O.deer(p, T, np.zeros(2), kind="dense", atol=1e-12)
    assert conv and iters == 1
    ref, _, _ = O.chain(p, T, np.zeros(2))
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-12)


def test_picard_and_newton_agree_with_each_other():
    """The J = 0 fixed-point iteration and DEER reach the same trace on tiny T (brute force)."""
    T = 12
    p, s0 = _problem("hmc_banana", T, seed=5)
    a, ia, ca, _ = O.deer(p, T, s0, kind="zero", atol=1e-12)
    b, ib, cb, _ = O.deer(p, T, s0, kind="dense", atol=1e-12)
    assert ca and cb and ia <= T and ib <= T
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10)


def test_step_rule_of_algorithm_1():
    T = 32
    p, s0 = _problem("mala_gauss", T)
    s, it, conv, _ = O.deer(p, T, s0, kind="dense", atol=1e-12, rule="step")
    ref, _, _ = O.chain(p, T, s0)
    assert conv
    np.testing.assert_allclose(s, ref, rtol=1e-10, atol=1e-10)


# ------------------------------------------------------------------------------------------
# Adjoint with decisions held
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("sp", [1.0, 1.6])
def test_adjoint_matches_frozen_finite_differences(sp):
    T, D = 40, 3
    t = small_logreg(N=30, D=D, sigma_p=sp)
    xi, u = W.noise(T, D, seed=6)
    eps = 0.03
    s0 = np.zeros(D)
    p = O.Problem(t, "mala", eps, xi=xi, u=u)
    s, _, acc = O.chain(p, T, s0)
    assert 0 < acc.mean() < 1
    dLds = 2.0 * s / T                     # L = mean_t |s_t|^2
    g = O.mala_adjoint(p, T, s0, s, acc, dLds)

    def L_of(e, spv):
        tt = O.Target("logreg", D, X=t.X, y=t.y, sigma_p=spv)
        pp = O.Problem(tt, "mala", e, xi=xi, u=u)
        ss = O.mala_chain_frozen(pp, T, s0, acc)
        return (ss ** 2).sum() / T

    h = 1e-4
    fd_e = (L_of(eps + h * eps, sp) - L_of(eps - h * eps, sp)) / (2 * h * eps)
    fd_s = (L_of(eps, sp + h) - L_of(eps, sp - h)) / (2 * h)
    assert g[0] == pytest.approx(fd_e, rel=1e-5)
    assert g[1] == pytest.approx(fd_s, rel=1e-5)
    # the frozen chain at the original parameters is the chain itself
    np.testing.assert_allclose(O.mala_chain_frozen(p, T, s0, acc), s, rtol=1e-14)


def test_non_finite_proposal_rejects_and_deer_does_not_stop_on_nan():
    """min(0, NaN) propagates NaN, so a divergent proposal rejects; a NaN iterate is never
    reported as converged, and Newton still reaches the trace in <= T updates."""
    t = O.Target("banana", 2)
    x = np.array([1e200, 1.0])
    out, dH, acc = O.hmc_step(t, 0.05, 4, x, np.array([0.1, 0.2]), 0.5)
    assert not acc and np.isnan(dH)
    np.testing.assert_array_equal(out, x)
    T = 60
    p, s0 = _problem("hmc_banana", T, seed=0)
    ref, _, _ = O.chain(p, T, s0)
    s, iters, conv, hist = O.deer(p, T, s0, kind="diag", atol=1e-10)   # undamped: blows up
    assert conv and iters <= T and not np.isnan(s).any()
    assert np.isinf(hist).any()
    np.testing.assert_allclose(s, ref, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("dense", [False, True])
def test_linear_recursion_is_sum_of_products(dense):
    """delta_t = sum_{k<=t} (A_t ... A_{k+1}) b_k, evaluated by explicit products."""
    rng = np.random.default_rng(3)
    T, n = 7, 3
    A = rng.standard_normal((T, n, n) if dense else (T, n))
    b = rng.standard_normal((T, n))
    got = O.linear_recursion(A, b, dense)
    for t in range(T):
        ref = np.zeros(n)
        for k in range(t + 1):
            M = np.eye(n)
            for j in range(k + 1, t + 1):
                M = (A[j] if dense else np.diag(A[j])) @ M
            ref += M @ b[k]
        np.testing.assert_allclose(got[t], ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------
# Reparameterised Gibbs on the hierarchical Gaussian (schools) model (Section 3.1, App. B.2)
# ------------------------------------------------------------------------------------------

# hyperparameters stated in Appendix B.2
_NU0, _TAU0SQ, _MU0, _KAPPA0, _ALPHA0, _SIGMA0SQ = 0.1, 100.0, 0.0, 0.1, 0.1, 10.0


def _log_inv_chi2(v, nu, s2):
    # scaled inverse chi-square(nu, s2) = inverse gamma(nu / 2, nu s2 / 2)
    return stats.invgamma.logpdf(v, a=nu / 2.0, scale=nu * s2 / 2.0)


def _schools_log_joint(tau2, mu, theta, sig2, X):
    """log p(tau^2, mu, theta, sigma^2, X) of the generative model, term by term (scipy)."""
    lp = _log_inv_chi2(tau2, _NU0, _TAU0SQ) + stats.norm.logpdf(mu, _MU0, np.sqrt(tau2 / _KAPPA0))
    lp = lp + np.sum([stats.norm.logpdf(th, mu, np.sqrt(tau2)) for th in theta], axis=0)
    lp = lp + np.sum([_log_inv_chi2(v, _ALPHA0, _SIGMA0SQ) for v in sig2], axis=0)
    for s in range(X.shape[0]):
        lp = lp + np.sum(stats.norm.logpdf(X[s][:, None], theta[s], np.sqrt(sig2[s])), axis=0)
    return lp


def _ks_against_density(draws, logdens, lo, hi, positive):
    """KS distance between the draws and the distribution whose log density (up to a constant)
    is logdens, integrated numerically on a fine grid over [lo, hi]."""
    grid = np.geomspace(lo, hi, 40001) if positive else np.linspace(lo, hi, 40001)
    lp = logdens(grid)
    w = np.exp(lp - lp.max())
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    x = np.sort(draws)
    F = np.interp(x, grid, cdf)
    n = len(x)
    return max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))


def test_gibbs_conditionals_match_the_joint_density():
    """Each coordinate update of the sweep, with the coordinates it conditions on held fixed and
    only its own noise varied, draws from the conditional that the model's joint density
    (scipy, term by term) gives by numerical integration: tau^2 | previous (mu, theta); mu |
    previous theta, new tau^2; theta_s | new (mu, tau^2), previous sigma^2_s; sigma^2_s | new
    theta_s.  This pins the conditionals, the order of the sweep and the reparameterisation
    noise (Inv-chi^2 base variates) together."""
    S, N, M = 3, 5, 4000
    X = W.schools_data(S, N, seed=4)
    D = 2 + 2 * S
    t = O.Target("schools", D, X=X)
    sp = W.schools_init(X) * np.array([1.3, 1.0] + [1.0] * S + [0.8] * S) + \
        np.array([0, 2.0] + [1.5] * S + [0] * S)
    base = W.gibbs_noise(1, S, N, seed=9)[0]
    pool = W.gibbs_noise(M, S, N, seed=10)
    crit = 1.95 / np.sqrt(M)  # KS critical value at p ~ 0.001

    def sweep_col(col, vary):
        out = []
        for m in range(M):
            xi = base.copy()
            xi[vary] = pool[m, vary]
            out.append(O.gibbs_sweep(t, sp, xi)[0][col])
        return np.array(out)

    th_p, sg_p = sp[2:2 + S], sp[2 + S:]
    fixed = O.gibbs_sweep(t, sp, base)[0]
    tau2_t, mu_t = fixed[0], fixed[1]
    # tau^2 | mu_{t-1}, theta_{t-1}
    d = sweep_col(0, 0)
    ks = _ks_against_density(d, lambda v: _schools_log_joint(v, sp[1], th_p, sg_p, X),
                             d.min() * 0.5, d.max() * 3.0, True)
    assert ks < crit, ("tau2", ks)
    # mu | theta_{t-1}, tau^2_t
    d = sweep_col(1, 1)
    span = d.max() - d.min()
    ks = _ks_against_density(d, lambda v: _schools_log_joint(tau2_t, v, th_p, sg_p, X),
                             d.min() - span, d.max() + span, False)
    assert ks < crit, ("mu", ks)
    for s in range(S):
        # theta_s | mu_t, tau^2_t, sigma^2_{s,t-1}
        d = sweep_col(2 + s, 2 + s)
        span = d.max() - d.min()

        def lth(v, s=s):
            th = [np.full_like(v, x) for x in th_p]
            th[s] = v
            return _schools_log_joint(tau2_t, mu_t, th, sg_p, X)
        ks = _ks_against_density(d, lth, d.min() - span, d.max() + span, False)
        assert ks < crit, ("theta", s, ks)
        # sigma^2_s | theta_{s,t}
        xi = base.copy()
        theta_t = O.gibbs_sweep(t, sp, xi)[0][2:2 + S]
        d = sweep_col(2 + S + s, 2 + S + s)

        def lsg(v, s=s):
            sg = [np.full_like(v, x) for x in sg_p]
            sg[s] = v
            return _schools_log_joint(tau2_t, mu_t, theta_t, sg, X)
        ks = _ks_against_density(d, lsg, d.min() * 0.5, d.max() * 3.0, True)
        assert ks < crit, ("sigma2", s, ks)


def test_gibbs_jacobian_matches_finite_differences():
    S, N = 4, 7
    X = W.schools_data(S, N, seed=2)
    D = 2 + 2 * S
    t = O.Target("schools", D, X=X)
    sp = W.schools_init(X)
    xi = W.gibbs_noise(1, S, N, seed=3)[0]
    _, J = O.gibbs_sweep(t, sp, xi)
    Jfd = np.zeros((D, D))
    for j in range(D):
        h = 1e-6 * (1 + abs(sp[j]))
        e = np.zeros(D)
        e[j] = h
        Jfd[:, j] = (O.gibbs_sweep(t, sp + e, xi)[0] - O.gibbs_sweep(t, sp - e, xi)[0]) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-8)
    # the sweep does not read the previous tau^2 (Eq. 6)
    assert np.all(J[:, 0] == 0.0)


@pytest.mark.parametrize("jac", ["dense", "diag"])
def test_gibbs_deer_reaches_sequential_trace(jac):
    S, N, T = 8, 20, 64
    X = W.schools_data(S, N)
    p = O.Problem(O.Target("schools", 2 + 2 * S, X=X), "gibbs", 0.0,
                  xi=W.gibbs_noise(T, S, N, seed=1), u=np.full(T, 0.5))
    s0 = W.schools_init(X)
    ref, _, acc = O.chain(p, T, s0)
    assert acc.all()
    s, iters, conv, _ = O.deer(p, T, s0, kind=jac, atol=1e-9, rtol=1e-12)
    assert conv and iters <= T
    np.testing.assert_allclose(s, ref, rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("jac", ["dense", "diag", "zero"])
def test_gibbs_deer_prefix_is_exact_after_k_iterations(jac):
    """After k Newton updates from s_t = s_0, the first k sweeps equal the sequential chain
    (Section 2's induction), for the Gibbs sweep as for the other samplers."""
    S, N, T = 4, 9, 30
    X = W.schools_data(S, N, seed=5)
    p = O.Problem(O.Target("schools", 2 + 2 * S, X=X), "gibbs", 0.0,
                  xi=W.gibbs_noise(T, S, N, seed=6), u=np.full(T, 0.5))
    s0 = W.schools_init(X)
    ref, _, _ = O.chain(p, T, s0)
    for k in range(1, 6):
        s, iters, _, _ = O.deer(p, T, s0, kind=jac, max_iters=k, atol=-1.0)
        assert iters == k
        np.testing.assert_allclose(s[:k], ref[:k], rtol=1e-11, atol=1e-11)


def test_gibbs_noise_distributions():
    """The Gibbs reparameterisation inputs: Inv-chi^2(nu, 1) base variates (scipy's inverse gamma
    with shape nu / 2 and scale nu / 2) for the variances, standard normals for the locations."""
    S, N, T = 5, 11, 20000
    xi = W.gibbs_noise(T, S, N, seed=3)
    nu_t, nu_s = 0.1 + S + 1, 0.1 + N
    crit = 1.95 / np.sqrt(T)
    assert stats.kstest(xi[:, 0], stats.invgamma(a=nu_t / 2, scale=nu_t / 2).cdf).statistic < crit
    for k in range(1, 2 + S):
        assert stats.kstest(xi[:, k], stats.norm.cdf).statistic < crit
    for k in range(2 + S, 2 + 2 * S):
        assert stats.kstest(xi[:, k], stats.invgamma(a=nu_s / 2, scale=nu_s / 2).cdf).statistic < crit
