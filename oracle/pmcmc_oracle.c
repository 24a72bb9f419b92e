/*
 * FP64 CPU oracle for "Parallelizing MCMC Across the Sequence Length" (arXiv 2508.18413).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  The CUDA library never calls it and shares no code,
 * header, table or constant with it.
 *
 * It is a plain, slow, sequential restatement of what the paper's samplers compute:
 *   - targets: Gaussian, Bayesian logistic regression, 2-D banana (log p, gradient, Hessian);
 *   - transitions f_t: MALA (Section 3.2), HMC with a sequential leapfrog (Algorithm 2), one
 *     leapfrog step on [x, v] (Eq. 7), MALA without the MH correction (ULA, for the affine
 *     special case of Section 2), and the reparameterised Gibbs sweep of the hierarchical
 *     Gaussian model (Section 3.1, Appendix B.2);
 *   - the sequential chain s_t = f_t(s_{t-1}) (Section 2), which is the exact answer;
 *   - the Newton Jacobians: the stop-gradient relaxation of the accept/reject gate
 *     (Section 3.2), its diagonal (quasi-DEER, Eq. 4), the leapfrog Jacobian (Eq. 8) and its
 *     block-diagonal form (block quasi-DEER, Appendix A.3);
 *   - a CPU DEER loop in the paper's own form (Eq. 3, Algorithm 1);
 *   - the adjoint of a chain functional with accept decisions held, and the frozen-decision
 *     chain used for finite differences;
 *   - Philox4x32-10 (Salmon et al., SC'11) and the noise counters, for the on-device noise row.
 *
 * Everything is double precision.  Dense matrices are row-major.  Parity status of each
 * function is recorded beside it ("pinned by": the independent check in tests/).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OT_GAUSSIAN 0
#define OT_LOGREG 1
#define OT_BANANA 2
#define OT_SCHOOLS 3

#define OS_MALA 0
#define OS_HMC 1
#define OS_LEAPFROG 2
#define OS_ULA 3
#define OS_GIBBS 4

#define OJ_DENSE 0
#define OJ_DIAG 1
#define OJ_BLOCK2 2
#define OJ_ZERO 4

typedef struct {
    int kind, D, N;
    const double *mu, *P; /* Gaussian N(mu, P^-1): mean (D), precision (D*D) */
    const double *X, *y;  /* logistic regression: design N*D, labels N; schools: scores S*N */
    double sigma_p;       /* logistic regression prior N(0, sigma_p^2 I) */
} o_target;

typedef struct {
    o_target tgt;
    int sampler;      /* OS_* */
    double eps;       /* step size */
    int L;            /* leapfrog steps per HMC transition */
    int gate_grad;    /* 1: Jacobian carries the stop-gradient gate term (Section 3.2) */
    double damping;   /* Newton Jacobian scaled by this factor (1 = none) */
    int clip;         /* 1: Newton Jacobian entries clipped to [-1, 1] after damping */
    const double *xi; /* T*D Gaussian noise (momentum for HMC) */
    const double *u;  /* T uniforms in (0, 1) */
} o_problem;

/* ---------------------------------------------------------------------------------------- */
/* Small dense helpers                                                                       */
/* ---------------------------------------------------------------------------------------- */

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* C = A B for n x n matrices */
static void matmul(int n, const double *A, const double *B, double *C) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double acc = 0.0;
            for (int k = 0; k < n; k++) acc += A[i * n + k] * B[k * n + j];
            C[i * n + j] = acc;
        }
}

/* y = A x (n x n) */
static void matvec(int n, const double *A, const double *x, double *y) {
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int k = 0; k < n; k++) acc += A[i * n + k] * x[k];
        y[i] = acc;
    }
}

/* y = A^T x (n x n) */
static void matTvec(int n, const double *A, const double *x, double *y) {
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int k = 0; k < n; k++) acc += A[k * n + i] * x[k];
        y[i] = acc;
    }
}

static double dot(int n, const double *a, const double *b) {
    double acc = 0.0;
    for (int i = 0; i < n; i++) acc += a[i] * b[i];
    return acc;
}

static double sigmoid(double z) {
    if (z >= 0) return 1.0 / (1.0 + exp(-z));
    double e = exp(z);
    return e / (1.0 + e);
}

/* log(1 + e^z), stable for both signs */
static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }

/* ---------------------------------------------------------------------------------------- */
/* Targets (L0).  Pinned by: FD of log p / gradient; scipy's multivariate normal log-density; */
/* sklearn/scipy Bernoulli log-likelihood; hand values of the banana formula.                */
/* ---------------------------------------------------------------------------------------- */

/* log p(x) up to an additive constant. */
double o_logp(const o_target *p, const double *x) {
    int D = p->D;
    if (p->kind == OT_GAUSSIAN) { /* -1/2 (x - mu)^T P (x - mu) */
        double acc = 0.0;
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++)
                acc += (x[i] - p->mu[i]) * p->P[i * D + j] * (x[j] - p->mu[j]);
        return -0.5 * acc;
    }
    if (p->kind == OT_LOGREG) { /* sum_n [y_n z_n - log(1 + e^{z_n})] - |x|^2 / (2 sigma_p^2) */
        double acc = 0.0;
        for (int n = 0; n < p->N; n++) {
            double z = dot(D, p->X + (size_t)n * D, x);
            acc += p->y[n] * z - softplus(z);
        }
        return acc - dot(D, x, x) / (2.0 * p->sigma_p * p->sigma_p);
    }
    /* banana: -x1^2/200 - (x2 + 0.1 x1^2 - 10)^2 / 2 */
    double b = x[1] + 0.1 * x[0] * x[0] - 10.0;
    return -x[0] * x[0] / 200.0 - 0.5 * b * b;
}

/* g = grad_x log p(x) */
void o_grad(const o_target *p, const double *x, double *g) {
    int D = p->D;
    if (p->kind == OT_GAUSSIAN) { /* -P (x - mu) */
        for (int i = 0; i < D; i++) {
            double acc = 0.0;
            for (int j = 0; j < D; j++) acc += p->P[i * D + j] * (x[j] - p->mu[j]);
            g[i] = -acc;
        }
        return;
    }
    if (p->kind == OT_LOGREG) { /* X^T (y - sigmoid(X x)) - x / sigma_p^2 */
        for (int d = 0; d < D; d++) g[d] = -x[d] / (p->sigma_p * p->sigma_p);
        for (int n = 0; n < p->N; n++) {
            const double *Xn = p->X + (size_t)n * D;
            double c = p->y[n] - sigmoid(dot(D, Xn, x));
            for (int d = 0; d < D; d++) g[d] += c * Xn[d];
        }
        return;
    }
    double b = x[1] + 0.1 * x[0] * x[0] - 10.0;
    g[0] = -x[0] / 100.0 - 0.2 * x[0] * b;
    g[1] = -b;
}

/* H = Hessian of log p at x (D x D) */
void o_hess(const o_target *p, const double *x, double *H) {
    int D = p->D;
    if (p->kind == OT_GAUSSIAN) {
        for (int i = 0; i < D * D; i++) H[i] = -p->P[i];
        return;
    }
    if (p->kind == OT_LOGREG) { /* -X^T diag(s(1-s)) X - I / sigma_p^2 */
        for (int i = 0; i < D * D; i++) H[i] = 0.0;
        for (int d = 0; d < D; d++) H[d * D + d] = -1.0 / (p->sigma_p * p->sigma_p);
        for (int n = 0; n < p->N; n++) {
            const double *Xn = p->X + (size_t)n * D;
            double s = sigmoid(dot(D, Xn, x));
            double w = s * (1.0 - s);
            for (int i = 0; i < D; i++)
                for (int j = 0; j < D; j++) H[i * D + j] -= w * Xn[i] * Xn[j];
        }
        return;
    }
    double b = x[1] + 0.1 * x[0] * x[0] - 10.0;
    H[0] = -0.01 - 0.04 * x[0] * x[0] - 0.2 * b;
    H[1] = -0.2 * x[0];
    H[2] = -0.2 * x[0];
    H[3] = -1.0;
}

/* ---------------------------------------------------------------------------------------- */
/* Transitions f_t (L1)                                                                      */
/* ---------------------------------------------------------------------------------------- */

int o_state_dim(const o_problem *pr) { return pr->sampler == OS_LEAPFROG ? 2 * pr->tgt.D : pr->tgt.D; }

/*
 * MALA transition (Section 3.2, the MALA function): proposal
 *   x~ = x + eps grad log p(x) + sqrt(2 eps) xi,
 * acceptance ratio p(x~) q(x | x~) / (p(x) q(x~ | x)) with q(a | b) = N(a; b + eps grad log p(b),
 * 2 eps I), gate g~ = log alpha - log u, accept iff g~ > 0.
 * Outputs: out = next state; *ell = log of the acceptance ratio before the min with 0;
 * *accept = decision.  With mh = 0 the proposal is returned unconditionally (ULA).
 * Pinned by: scipy normal log-densities for q; Gaussian moments of a long chain.
 */
void o_mala_step(const o_target *tg, double eps, const double *x, const double *xi, double u,
                 int mh, double *out, double *ell, int *accept) {
    int D = tg->D;
    double *g = dalloc(D), *xt = dalloc(D), *gt = dalloc(D);
    o_grad(tg, x, g);
    for (int d = 0; d < D; d++) xt[d] = x[d] + eps * g[d] + sqrt(2.0 * eps) * xi[d];
    if (!mh) {
        memcpy(out, xt, sizeof(double) * D);
        if (ell) *ell = 0.0;
        if (accept) *accept = 1;
        free(g); free(xt); free(gt);
        return;
    }
    o_grad(tg, xt, gt);
    double lq_fwd = 0.0, lq_rev = 0.0; /* log q(x~ | x) and log q(x | x~), up to constants */
    for (int d = 0; d < D; d++) {
        double a = xt[d] - x[d] - eps * g[d];
        double b = x[d] - xt[d] - eps * gt[d];
        lq_fwd += a * a;
        lq_rev += b * b;
    }
    lq_fwd = -lq_fwd / (4.0 * eps);
    lq_rev = -lq_rev / (4.0 * eps);
    double l = o_logp(tg, xt) - o_logp(tg, x) + lq_rev - lq_fwd;
    /* min(0, l) propagating NaN, so a non-finite ratio (a divergent proposal) rejects */
    double log_alpha = (l < 0.0 || isnan(l)) ? l : 0.0;
    double gtilde = log_alpha - log(u);
    int acc = gtilde > 0.0;
    memcpy(out, acc ? xt : x, sizeof(double) * D);
    if (ell) *ell = l;
    if (accept) *accept = acc;
    free(g); free(xt); free(gt);
}

/*
 * HMC transition with a sequential leapfrog (Algorithm 2, with x0 = the previous state and the
 * momentum v0 = xi):  H0 = |v0|^2/2 - log p(x0); half step on v; L steps
 * x += eps v, v += eps grad log p(x); negative half step on v; HL = |vL|^2/2 - log p(xL).
 * The accept test printed in Algorithm 2 is garbled; this follows the standard Metropolis rule
 * it stands for: log alpha = min(0, H0 - HL), accept iff log alpha - log u > 0.
 * *dH = H0 - HL.  Pinned by: Gaussian and banana moments of long chains; leapfrog reversibility.
 */
void o_hmc_step(const o_target *tg, double eps, int L, const double *x0, const double *xi,
                double u, double *out, double *dH, int *accept) {
    int D = tg->D;
    double *x = dalloc(D), *v = dalloc(D), *g = dalloc(D);
    memcpy(x, x0, sizeof(double) * D);
    memcpy(v, xi, sizeof(double) * D);
    double H0 = 0.5 * dot(D, v, v) - o_logp(tg, x);
    o_grad(tg, x, g);
    for (int d = 0; d < D; d++) v[d] += 0.5 * eps * g[d];
    for (int k = 0; k < L; k++) {
        for (int d = 0; d < D; d++) x[d] += eps * v[d];
        o_grad(tg, x, g);
        for (int d = 0; d < D; d++) v[d] += eps * g[d];
    }
    for (int d = 0; d < D; d++) v[d] -= 0.5 * eps * g[d];
    double HL = 0.5 * dot(D, v, v) - o_logp(tg, x);
    double diff = H0 - HL;
    double log_alpha = (diff < 0.0 || isnan(diff)) ? diff : 0.0; /* NaN rejects */
    int acc = (log_alpha - log(u)) > 0.0;
    memcpy(out, acc ? x : x0, sizeof(double) * D);
    if (dH) *dH = diff;
    if (accept) *accept = acc;
    free(x); free(v); free(g);
}

/* One leapfrog step on s = [x, v] (Eq. 7): x' = x + eps v;  v' = v + eps grad log p(x'). */
void o_leapfrog(const o_target *tg, double eps, const double *s, double *out) {
    int D = tg->D;
    double *g = dalloc(D);
    for (int d = 0; d < D; d++) out[d] = s[d] + eps * s[D + d];
    o_grad(tg, out, g);
    for (int d = 0; d < D; d++) out[D + d] = s[D + d] + eps * g[d];
    free(g);
}

/*
 * Reparameterised Gibbs sweep of the hierarchical Gaussian ("eight schools") model of the Gibbs
 * experiment (Section 3.1, Eq. 5-6; the model, its hyperparameters and the coordinate order are
 * those of Appendix B.2).  S schools with N scores each, X[s*N + n]; state
 *   s = (tau^2, mu, theta_1..theta_S, sigma^2_1..sigma^2_S),  D = 2 + 2S.
 * Model: tau^2 ~ Inv-chi^2(nu0, tau0^2), mu | tau^2 ~ N(mu0, tau^2 / kappa0),
 * theta_s | mu, tau^2 ~ N(mu, tau^2), sigma^2_s ~ Inv-chi^2(alpha0, sigma0^2),
 * x_sn | theta_s, sigma^2_s ~ N(theta_s, sigma^2_s)  (Inv-chi^2 = scaled inverse chi-square).
 * Conjugacy gives the conditionals used in order:
 *   tau^2   | mu, theta            Inv-chi^2(nu0 + S + 1, A / (nu0 + S + 1)),
 *                                  A = nu0 tau0^2 + kappa0 (mu - mu0)^2 + sum_s (theta_s - mu)^2;
 *   mu      | theta, tau^2         N((kappa0 mu0 + sum_s theta_s) / (kappa0 + S), tau^2 / (kappa0 + S));
 *   theta_s | mu, tau^2, sigma^2_s N(m_s, 1 / P_s),  P_s = 1 / tau^2 + N / sigma^2_s,
 *                                  m_s = (mu / tau^2 + sum_n x_sn / sigma^2_s) / P_s;
 *   sigma^2_s | theta_s            Inv-chi^2(alpha0 + N, B_s / (alpha0 + N)),
 *                                  B_s = alpha0 sigma0^2 + sum_n (x_sn - theta_s)^2;
 * tau^2 and mu use the previous sweep's theta and mu, theta_s the previous sigma^2_s, so the sweep
 * does not depend on the previous tau^2 (Eq. 6).  Reparameterisation: the noise xi (D values) holds
 * xi[0] ~ Inv-chi^2(nu0 + S + 1, 1), xi[1] and xi[2 + s] ~ N(0, 1), xi[2 + S + s] ~
 * Inv-chi^2(alpha0 + N, 1); an Inv-chi^2(nu, 1) variate times c is Inv-chi^2(nu, c) (Appendix B.2),
 * a standard normal times sd plus mean is N(mean, sd^2).
 * J (may be NULL): the D x D Jacobian d out / d s_prev, row by row in the order of the updates
 * (forward-mode chain rule through the sweep).
 * Pinned by: each conditional's draws against scipy's distributions (tests/test_oracle.py),
 * finite differences of J, zero first column of J.
 */
#define SCH_NU0 0.1
#define SCH_TAU0SQ 100.0
#define SCH_MU0 0.0
#define SCH_KAPPA0 0.1
#define SCH_ALPHA0 0.1
#define SCH_SIGMA0SQ 10.0

void o_gibbs_sweep(const o_target *tg, const double *sp, const double *xi, double *out, double *J) {
    int D = tg->D, S = (D - 2) / 2, N = tg->N;
    const double *X = tg->X;
    double *dtau = dalloc(D), *dmu = dalloc(D), *dth = dalloc(D), *dP = dalloc(D), *da = dalloc(D);
    double mu_p = sp[1];
    /* tau^2 */
    double nu_n = SCH_NU0 + S + 1, A = SCH_NU0 * SCH_TAU0SQ + SCH_KAPPA0 * (mu_p - SCH_MU0) * (mu_p - SCH_MU0);
    double sum_dev = 0.0, sum_th = 0.0;
    for (int k = 0; k < S; k++) {
        double dv = sp[2 + k] - mu_p;
        A += dv * dv;
        sum_dev += dv;
        sum_th += sp[2 + k];
    }
    double tau2 = xi[0] * A / nu_n;
    out[0] = tau2;
    dtau[1] = xi[0] / nu_n * (2.0 * SCH_KAPPA0 * (mu_p - SCH_MU0) - 2.0 * sum_dev);
    for (int k = 0; k < S; k++) dtau[2 + k] = xi[0] / nu_n * 2.0 * (sp[2 + k] - mu_p);
    /* mu */
    double kS = SCH_KAPPA0 + S;
    double mu = (SCH_KAPPA0 * SCH_MU0 + sum_th) / kS + sqrt(tau2 / kS) * xi[1];
    out[1] = mu;
    double c_mu = xi[1] / (2.0 * sqrt(kS * tau2));
    for (int j = 0; j < D; j++) dmu[j] = c_mu * dtau[j];
    for (int k = 0; k < S; k++) dmu[2 + k] += 1.0 / kS;
    if (J) {
        for (int j = 0; j < D; j++) {
            J[0 * D + j] = dtau[j];
            J[1 * D + j] = dmu[j];
        }
    }
    /* theta_s, then sigma^2_s */
    for (int k = 0; k < S; k++) {
        double sg = sp[2 + S + k], sx = 0.0;
        for (int n = 0; n < N; n++) sx += X[(size_t)k * N + n];
        double P = 1.0 / tau2 + N / sg;
        double a = mu / tau2 + sx / sg;
        double m = a / P;
        double th = m + xi[2 + k] / sqrt(P);
        out[2 + k] = th;
        double B = SCH_ALPHA0 * SCH_SIGMA0SQ, dB = 0.0;
        for (int n = 0; n < N; n++) {
            double e = X[(size_t)k * N + n] - th;
            B += e * e;
            dB += -2.0 * e;
        }
        double an = SCH_ALPHA0 + N;
        out[2 + S + k] = xi[2 + S + k] * B / an;
        if (J) {
            for (int j = 0; j < D; j++) {
                dP[j] = -dtau[j] / (tau2 * tau2);
                da[j] = dmu[j] / tau2 - mu * dtau[j] / (tau2 * tau2);
            }
            dP[2 + S + k] += -N / (sg * sg);
            da[2 + S + k] += -sx / (sg * sg);
            for (int j = 0; j < D; j++) {
                double dm = da[j] / P - a * dP[j] / (P * P);
                dth[j] = dm - 0.5 * xi[2 + k] * dP[j] / (P * sqrt(P));
                J[(2 + k) * D + j] = dth[j];
                J[(2 + S + k) * D + j] = xi[2 + S + k] / an * dB * dth[j];
            }
        }
    }
    free(dtau); free(dmu); free(dth); free(dP); free(da);
}

/* f_t(s_prev) for the problem's sampler; t is 1-based.  *ell: MALA log ratio / HMC H0-HL. */
void o_f(const o_problem *pr, int t, const double *s_prev, double *out, double *ell, int *accept) {
    int D = pr->tgt.D;
    const double *xi = pr->xi ? pr->xi + (size_t)(t - 1) * D : NULL;
    double u = pr->u ? pr->u[t - 1] : 0.5;
    switch (pr->sampler) {
    case OS_MALA: o_mala_step(&pr->tgt, pr->eps, s_prev, xi, u, 1, out, ell, accept); break;
    case OS_ULA: o_mala_step(&pr->tgt, pr->eps, s_prev, xi, u, 0, out, ell, accept); break;
    case OS_HMC: o_hmc_step(&pr->tgt, pr->eps, pr->L, s_prev, xi, u, out, ell, accept); break;
    case OS_GIBBS:
        o_gibbs_sweep(&pr->tgt, s_prev, xi, out, NULL);
        if (ell) *ell = 0.0;
        if (accept) *accept = 1;
        break;
    default:
        o_leapfrog(&pr->tgt, pr->eps, s_prev, out);
        if (ell) *ell = 0.0;
        if (accept) *accept = 1;
    }
}

/*
 * The sequential chain s_t = f_t(s_{t-1}), t = 1..T (Section 2).  This is the exact answer the
 * parallel Newton solve must reach (Section 3.2: "the same set of samples up to the numerical
 * tolerance").  s: T*n output; ell, accept: per-step MH quantities (may be NULL).
 */
void o_chain(const o_problem *pr, int T, const double *s0, double *s, double *ell, int *accept) {
    int n = o_state_dim(pr);
    for (int t = 1; t <= T; t++) {
        const double *prev = t == 1 ? s0 : s + (size_t)(t - 2) * n;
        o_f(pr, t, prev, s + (size_t)(t - 1) * n, ell ? ell + t - 1 : NULL,
            accept ? accept + t - 1 : NULL);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* Newton Jacobians (L2)                                                                     */
/* ---------------------------------------------------------------------------------------- */

static double dsigmoid(double z) {
    double s = sigmoid(z);
    return s * (1.0 - s);
}

/*
 * Jacobian of the MALA transition under the stop-gradient gate of Section 3.2:
 * x_t = g x~ + (1 - g) x with g = sigma(g~) + stop_gradient(1(g~ > 0) - sigma(g~)).  Its value
 * is the indicator; its derivative is sigma'(g~) grad g~.  Hence
 *   J = g (I + eps H(x)) + (1 - g) I + sigma'(g~) (x~ - x) (grad g~)^T,
 * grad g~ = grad min(0, ell) = 1(ell < 0) grad ell (zero at ell >= 0), and, with
 * A = I + eps H(x), B = I + eps H(x~), e = x - x~ - eps grad log p(x~) (log q(x~|x) does not
 * depend on x once xi is fixed):
 *   grad ell = A^T grad log p(x~) - grad log p(x) - (1 / (2 eps)) (I - B A)^T e.
 * gate_grad = 0 drops the sigma' term (gate held).
 * Pinned by: central finite differences of the relaxed map sigma(g~) x~ + (1 - sigma(g~)) x.
 */
void o_mala_jac(const o_target *tg, double eps, const double *x, const double *xi, double u,
                int gate_grad, double *J) {
    int D = tg->D;
    double *g = dalloc(D), *xt = dalloc(D), *gt = dalloc(D), *e = dalloc(D);
    double *A = dalloc((size_t)D * D), *B = dalloc((size_t)D * D), *BA = dalloc((size_t)D * D);
    double *gell = dalloc(D), *tmp = dalloc(D);
    double ell;
    int acc;
    double *xn = dalloc(D);
    o_mala_step(tg, eps, x, xi, u, 1, xn, &ell, &acc);
    o_grad(tg, x, g);
    for (int d = 0; d < D; d++) xt[d] = x[d] + eps * g[d] + sqrt(2.0 * eps) * xi[d];
    o_grad(tg, xt, gt);
    o_hess(tg, x, A);
    o_hess(tg, xt, B);
    for (int i = 0; i < D * D; i++) { A[i] *= eps; B[i] *= eps; }
    for (int d = 0; d < D; d++) { A[d * D + d] += 1.0; B[d * D + d] += 1.0; }
    double gv = acc ? 1.0 : 0.0;
    for (int i = 0; i < D; i++)
        for (int j = 0; j < D; j++) J[i * D + j] = gv * A[i * D + j] + (i == j ? 1.0 - gv : 0.0);
    if (gate_grad && ell < 0.0) {
        double gtilde = ell - log(u);
        for (int d = 0; d < D; d++) e[d] = x[d] - xt[d] - eps * gt[d];
        matTvec(D, A, gt, gell);                  /* A^T grad log p(x~) */
        matmul(D, B, A, BA);
        for (int i = 0; i < D * D; i++) BA[i] = -BA[i];
        for (int d = 0; d < D; d++) BA[d * D + d] += 1.0; /* I - B A */
        matTvec(D, BA, e, tmp);
        for (int d = 0; d < D; d++) gell[d] = gell[d] - g[d] - tmp[d] / (2.0 * eps);
        double c = dsigmoid(gtilde);
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) J[i * D + j] += c * (xt[i] - x[i]) * gell[j];
    }
    free(g); free(xt); free(gt); free(e); free(A); free(B); free(BA); free(gell); free(tmp);
    free(xn);
}

/*
 * Jacobian of the HMC transition under the same stop-gradient gate:
 *   J = g M_x + (1 - g) I + sigma'(g~) (x_L - x_0) (grad g~)^T,
 * M_x = d x_L / d x_0, and, with M_v = d v_L / d x_0 (v_0 = xi does not depend on x_0),
 *   grad g~ = 1(H0 - HL < 0) [ -grad log p(x_0) - M_v^T v_L + M_x^T grad log p(x_L) ].
 * M_x and M_v are carried through the leapfrog as dense tangents.
 * Pinned by: central finite differences of the relaxed map.
 */
void o_hmc_jac(const o_target *tg, double eps, int L, const double *x0, const double *xi,
               double u, int gate_grad, double *J) {
    int D = tg->D;
    size_t DD = (size_t)D * D;
    double *x = dalloc(D), *v = dalloc(D), *g = dalloc(D), *g0 = dalloc(D);
    double *Mx = dalloc(DD), *Mv = dalloc(DD), *H = dalloc(DD), *HM = dalloc(DD);
    double *gH = dalloc(D), *tmp = dalloc(D);
    memcpy(x, x0, sizeof(double) * D);
    memcpy(v, xi, sizeof(double) * D);
    double H0 = 0.5 * dot(D, v, v) - o_logp(tg, x);
    o_grad(tg, x, g0);
    for (int d = 0; d < D; d++) v[d] += 0.5 * eps * g0[d];
    for (int d = 0; d < D; d++) Mx[d * D + d] = 1.0;
    o_hess(tg, x, H);
    for (size_t i = 0; i < DD; i++) Mv[i] = 0.5 * eps * H[i];
    for (int k = 0; k < L; k++) {
        for (int d = 0; d < D; d++) x[d] += eps * v[d];
        for (size_t i = 0; i < DD; i++) Mx[i] += eps * Mv[i];
        o_grad(tg, x, g);
        for (int d = 0; d < D; d++) v[d] += eps * g[d];
        o_hess(tg, x, H);
        matmul(D, H, Mx, HM);
        for (size_t i = 0; i < DD; i++) Mv[i] += eps * HM[i];
    }
    for (int d = 0; d < D; d++) v[d] -= 0.5 * eps * g[d];
    o_hess(tg, x, H);
    matmul(D, H, Mx, HM);
    for (size_t i = 0; i < DD; i++) Mv[i] -= 0.5 * eps * HM[i];
    double HL = 0.5 * dot(D, v, v) - o_logp(tg, x);
    double diff = H0 - HL;
    double log_alpha = (diff < 0.0 || isnan(diff)) ? diff : 0.0;
    double gtilde = log_alpha - log(u);
    double gv = gtilde > 0.0 ? 1.0 : 0.0;
    for (int i = 0; i < D; i++)
        for (int j = 0; j < D; j++) J[i * D + j] = gv * Mx[i * D + j] + (i == j ? 1.0 - gv : 0.0);
    if (gate_grad && diff < 0.0) {
        matTvec(D, Mv, v, tmp);
        matTvec(D, Mx, g, gH); /* g = grad log p(x_L) */
        for (int d = 0; d < D; d++) gH[d] = -g0[d] - tmp[d] + gH[d];
        double c = dsigmoid(gtilde);
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) J[i * D + j] += c * (x[i] - x0[i]) * gH[j];
    }
    free(x); free(v); free(g); free(g0); free(Mx); free(Mv); free(H); free(HM); free(gH);
    free(tmp);
}

/*
 * Leapfrog Jacobian (Eq. 8): [[I, eps I], [eps H(x'), I + eps^2 H(x')]] with x' = x + eps v.
 * Pinned by: central finite differences of o_leapfrog.
 */
void o_leapfrog_jac(const o_target *tg, double eps, const double *s, double *J) {
    int D = tg->D, n = 2 * D;
    double *xp = dalloc(D), *H = dalloc((size_t)D * D);
    for (int d = 0; d < D; d++) xp[d] = s[d] + eps * s[D + d];
    o_hess(tg, xp, H);
    for (int i = 0; i < n * n; i++) J[i] = 0.0;
    for (int i = 0; i < D; i++) {
        J[i * n + i] = 1.0;
        J[i * n + D + i] = eps;
        for (int j = 0; j < D; j++) {
            J[(D + i) * n + j] = eps * H[i * D + j];
            J[(D + i) * n + D + j] = eps * eps * H[i * D + j] + (i == j ? 1.0 : 0.0);
        }
    }
    free(xp); free(H);
}

/*
 * Newton Jacobian of kind `kind` at s_prev, as a dense n x n matrix:
 *   OJ_DENSE  the full Jacobian (DEER, Eq. 2);
 *   OJ_DIAG   its diagonal (quasi-DEER, Eq. 4);
 *   OJ_BLOCK2 the diagonal of each D x D block (block quasi-DEER, Appendix A.3);
 *   OJ_ZERO   zero (the fixed-point / Picard-type iteration s_t <- f_t(s_{t-1})).
 * Then J <- damping J and, if clip, each entry clipped to [-1, 1] (Appendix B.4).
 */
void o_jac(const o_problem *pr, int t, const double *s_prev, int kind, double *J) {
    int D = pr->tgt.D, n = o_state_dim(pr);
    const double *xi = pr->xi ? pr->xi + (size_t)(t - 1) * D : NULL;
    double u = pr->u ? pr->u[t - 1] : 0.5;
    if (kind == OJ_ZERO) {
        for (int i = 0; i < n * n; i++) J[i] = 0.0;
        return;
    }
    switch (pr->sampler) {
    case OS_MALA: o_mala_jac(&pr->tgt, pr->eps, s_prev, xi, u, pr->gate_grad, J); break;
    case OS_HMC: o_hmc_jac(&pr->tgt, pr->eps, pr->L, s_prev, xi, u, pr->gate_grad, J); break;
    case OS_LEAPFROG: o_leapfrog_jac(&pr->tgt, pr->eps, s_prev, J); break;
    case OS_GIBBS: {
        double *tmp = dalloc(n);
        o_gibbs_sweep(&pr->tgt, s_prev, xi, tmp, J);
        free(tmp);
        break;
    }
    default: { /* ULA: I + eps H(x) */
        o_hess(&pr->tgt, s_prev, J);
        for (int i = 0; i < D * D; i++) J[i] *= pr->eps;
        for (int d = 0; d < D; d++) J[d * D + d] += 1.0;
    }
    }
    if (kind == OJ_DIAG) {
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if (i != j) J[i * n + j] = 0.0;
    } else if (kind == OJ_BLOCK2) {
        int h = n / 2;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if ((i % h) != (j % h)) J[i * n + j] = 0.0;
    }
    for (int i = 0; i < n * n; i++) {
        J[i] *= pr->damping;
        if (pr->clip) J[i] = J[i] > 1.0 ? 1.0 : (J[i] < -1.0 ? -1.0 : J[i]);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* DEER (Eqs. 1-3, Algorithm 1), sequential CPU form                                         */
/* ---------------------------------------------------------------------------------------- */

/*
 * Newton iterations for the fixed point of s_t = f_t(s_{t-1}).
 * Each iteration evaluates f_t and J_t at the previous iterate for all t, forms
 *   u_t = f_t(s^(i)_{t-1}) - J_t s^(i)_{t-1}                       (Eq. 3)
 * and solves the linear recursion s^(i+1)_t = J_t s^(i+1)_{t-1} + u_t from s_0, here by the plain
 * sequential loop (the parallel machine would use a scan; the result is the same).
 * Stopping (rule 0): the residual of Eq. 1, max_{t,d} (|s_t - f_t(s_{t-1})| - rtol |s_t|) <= atol,
 * checked on the current iterate before the update; that iterate is returned.
 * Stopping (rule 1): Algorithm 1's step size, max_t |s^(i+1)_t - s^(i)_t|_inf <= atol; the new
 * iterate is returned.
 * s_init: T*n initial guess (NULL: s_t = s_0 for all t).  s_out: T*n result.
 * hist (may be NULL, max_iters + 1 entries): max_t,d |residual| of each evaluated iterate.
 * Returns the number of Newton updates applied; *converged set to 1 when the rule was met.
 */
int o_deer(const o_problem *pr, int kind, int T, const double *s0, const double *s_init,
           int max_iters, double atol, double rtol, int rule, double *s_out, double *hist,
           int *converged) {
    int n = o_state_dim(pr);
    size_t nn = (size_t)n * n;
    double *s = s_out;
    double *f = dalloc((size_t)T * n), *J = dalloc((size_t)T * nn), *uu = dalloc((size_t)T * n);
    double *snew = dalloc((size_t)T * n), *tmp = dalloc(n);
    for (int t = 0; t < T; t++)
        for (int d = 0; d < n; d++) s[(size_t)t * n + d] = s_init ? s_init[(size_t)t * n + d] : s0[d];
    int it = 0;
    *converged = 0;
    for (;;) {
        double err = -INFINITY, rmax = 0.0;
        for (int t = 1; t <= T; t++) {
            const double *prev = t == 1 ? s0 : s + (size_t)(t - 2) * n;
            o_f(pr, t, prev, f + (size_t)(t - 1) * n, NULL, NULL);
            for (int d = 0; d < n; d++) {
                double st = s[(size_t)(t - 1) * n + d];
                double r = fabs(st - f[(size_t)(t - 1) * n + d]);
                double e = r - rtol * fabs(st);
                if (isnan(e)) r = e = INFINITY; /* a non-finite iterate is not converged */
                if (r > rmax) rmax = r;
                if (e > err) err = e;
            }
        }
        if (hist) hist[it] = rmax;
        if (rule == 0 && err <= atol) { *converged = 1; break; }
        if (it >= max_iters) break;
        for (int t = 1; t <= T; t++) {
            const double *prev = t == 1 ? s0 : s + (size_t)(t - 2) * n;
            double *Jt = J + (size_t)(t - 1) * nn;
            o_jac(pr, t, prev, kind, Jt);
            matvec(n, Jt, prev, tmp);
            for (int d = 0; d < n; d++) uu[(size_t)(t - 1) * n + d] = f[(size_t)(t - 1) * n + d] - tmp[d];
        }
        double dmax = 0.0;
        for (int t = 1; t <= T; t++) {
            const double *prev = t == 1 ? s0 : snew + (size_t)(t - 2) * n;
            matvec(n, J + (size_t)(t - 1) * nn, prev, tmp);
            for (int d = 0; d < n; d++) {
                double v = tmp[d] + uu[(size_t)(t - 1) * n + d];
                snew[(size_t)(t - 1) * n + d] = v;
                double dd = fabs(v - s[(size_t)(t - 1) * n + d]);
                if (dd > dmax) dmax = dd;
            }
        }
        memcpy(s, snew, sizeof(double) * (size_t)T * n);
        it++;
        if (rule == 1 && dmax <= atol) { *converged = 1; break; }
    }
    free(f); free(J); free(uu); free(snew); free(tmp);
    return it;
}

/* ---------------------------------------------------------------------------------------- */
/* Adjoint of a chain functional with the accept decisions held                              */
/* ---------------------------------------------------------------------------------------- */

/*
 * MALA chain with every accept decision frozen to acc[t]: s_t = acc_t ? x~(s_{t-1}) : s_{t-1}.
 * With the decisions held, the chain is a smooth function of (eps, sigma_p); this is the map
 * the finite-difference check differentiates.
 */
void o_mala_chain_frozen(const o_problem *pr, int T, const double *s0, const int *acc, double *s) {
    int D = pr->tgt.D;
    double *g = dalloc(D);
    for (int t = 1; t <= T; t++) {
        const double *x = t == 1 ? s0 : s + (size_t)(t - 2) * D;
        double *out = s + (size_t)(t - 1) * D;
        if (acc[t - 1]) {
            const double *xi = pr->xi + (size_t)(t - 1) * D;
            o_grad(&pr->tgt, x, g);
            for (int d = 0; d < D; d++) out[d] = x[d] + pr->eps * g[d] + sqrt(2.0 * pr->eps) * xi[d];
        } else {
            memmove(out, x, sizeof(double) * D);
        }
    }
    free(g);
}

/*
 * Gradient of a chain functional L(s_1..s_T) with respect to theta = (eps, sigma_p) for MALA
 * with the accept decisions held: the reverse recursion
 *   lambda_T = dL/ds_T,  lambda_t = dL/ds_t + J_{t+1}^T lambda_{t+1},
 *   dL/dtheta = sum_t lambda_t^T d f_t / d theta,
 * with J_{t+1} = I + eps H(s_t) when step t+1 was accepted and I otherwise, and, for an
 * accepted step from x = s_{t-1}:  d f/d eps = grad log p(x) + xi_t / sqrt(2 eps),
 * d f / d sigma_p = eps * 2 x / sigma_p^3 (logistic target; zero for the others).
 * dLds: T*D.  grad[0] = dL/d eps, grad[1] = dL/d sigma_p.
 * Pinned by: central finite differences of o_mala_chain_frozen.
 */
void o_mala_adjoint(const o_problem *pr, int T, const double *s0, const double *s, const int *acc,
                    const double *dLds, double *grad) {
    int D = pr->tgt.D;
    double *lam = dalloc(D), *tmp = dalloc(D), *H = dalloc((size_t)D * D), *g = dalloc(D);
    grad[0] = grad[1] = 0.0;
    for (int t = T; t >= 1; t--) {
        /* lambda_t = dL/ds_t + J_{t+1}^T lambda_{t+1} */
        if (t < T && acc[t]) { /* step t+1 accepted: J = I + eps H(s_t), symmetric */
            o_hess(&pr->tgt, s + (size_t)(t - 1) * D, H);
            matTvec(D, H, lam, tmp);
            for (int d = 0; d < D; d++) lam[d] += pr->eps * tmp[d];
        }
        for (int d = 0; d < D; d++) lam[d] += dLds[(size_t)(t - 1) * D + d];
        if (acc[t - 1]) {
            const double *x = t == 1 ? s0 : s + (size_t)(t - 2) * D;
            const double *xi = pr->xi + (size_t)(t - 1) * D;
            o_grad(&pr->tgt, x, g);
            for (int d = 0; d < D; d++) {
                grad[0] += lam[d] * (g[d] + xi[d] / sqrt(2.0 * pr->eps));
                if (pr->tgt.kind == OT_LOGREG) {
                    double sp = pr->tgt.sigma_p;
                    grad[1] += lam[d] * pr->eps * 2.0 * x[d] / (sp * sp * sp);
                }
            }
        }
    }
    free(lam); free(tmp); free(H); free(g);
}

/* ---------------------------------------------------------------------------------------- */
/* Philox4x32-10 and the noise counters                                                      */
/* ---------------------------------------------------------------------------------------- */

/*
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): ten rounds of the 4x32 S-P network with multipliers 0xD2511F53 and 0xCD9E8D57 and
 * the key schedule bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
 * Pinned by: the published known-answer vectors.
 */
void o_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform on the open interval (0, 1) from a 64-bit word: (k + 1/2) 2^-53 */
static double u53(uint32_t lo, uint32_t hi) {
    uint64_t k = (((uint64_t)hi << 32) | lo) >> 11;
    return ((double)k + 0.5) * (1.0 / 9007199254740992.0);
}

/*
 * Noise of chain `chain` from a 64-bit seed (key = (low word, high word)), t = 1..T:
 *   xi[t][2j], xi[t][2j+1]: Box-Muller of the two uniforms from counter (j, t-1, chain, 0);
 *   u[t]: the first uniform from counter (0, t-1, chain, 1).
 * Box-Muller: r = sqrt(-2 log u1), theta = 2 pi u2, (r cos theta, r sin theta).
 * raw (may be NULL): T * ceil(D/2) * 4 words of stream 0 followed by T * 4 words of stream 1.
 */
void o_gen_noise(uint64_t seed, uint32_t chain, int T, int D, double *xi, double *u, uint32_t *raw) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int P = (D + 1) / 2;
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 1; t <= T; t++) {
        for (int j = 0; j < P; j++) {
            uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(t - 1), chain, 0u}, w[4];
            o_philox4x32_10(ctr, key, w);
            if (raw) memcpy(raw + ((size_t)(t - 1) * P + j) * 4, w, sizeof(w));
            double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
            double r = sqrt(-2.0 * log(u1)), th = two_pi * u2;
            xi[(size_t)(t - 1) * D + 2 * j] = r * cos(th);
            if (2 * j + 1 < D) xi[(size_t)(t - 1) * D + 2 * j + 1] = r * sin(th);
        }
        uint32_t ctr[4] = {0u, (uint32_t)(t - 1), chain, 1u}, w[4];
        o_philox4x32_10(ctr, key, w);
        if (raw) memcpy(raw + (size_t)T * P * 4 + (size_t)(t - 1) * 4, w, sizeof(w));
        u[t - 1] = u53(w[0], w[1]);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* The linear recursion solved by each Newton iteration (Section 2, in delta form)            */
/* ---------------------------------------------------------------------------------------- */

/*
 * delta_t = A_t delta_{t-1} + b_t for t = 0..T-1 with delta_{-1} = 0, written out as the plain
 * sequential loop (the definition the parallel scan must reproduce).
 * dense = 0: A is T*n (elementwise maps); dense = 1: A is T*n*n row-major.
 * Pinned by: brute-force sums of products of the maps on tiny inputs.
 */
void o_linear_recursion(int T, int n, int dense, const double *A, const double *b, double *delta) {
    double *prev = dalloc(n), *tmp = dalloc(n);
    for (int t = 0; t < T; t++) {
        if (dense)
            matvec(n, A + (size_t)t * n * n, prev, tmp);
        else
            for (int d = 0; d < n; d++) tmp[d] = A[(size_t)t * n + d] * prev[d];
        for (int d = 0; d < n; d++) {
            prev[d] = tmp[d] + b[(size_t)t * n + d];
            delta[(size_t)t * n + d] = prev[d];
        }
    }
    free(prev); free(tmp);
}
