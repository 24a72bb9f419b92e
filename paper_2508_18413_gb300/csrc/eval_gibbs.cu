// Reparameterised Gibbs sampling of the hierarchical Gaussian ("schools") model: evaluate and
// linearise f_t at every t (step (a) of a Newton iteration), and the sequential chain.
//
// Section 3.1 writes a Gibbs sweep as a deterministic, differentiable function of the previous
// state and per-sweep noise, x_t = f(x_{t-1}, xi_t) (Eq. 5), composed of one update per
// coordinate, each conditioned on the newest values of the others (Eq. 6).  The model and the
// order of its updates are those of the Gibbs experiment (Appendix B.2): S schools of N scores,
//   tau^2 ~ Inv-chi^2(nu0, tau0^2),  mu | tau^2 ~ N(mu0, tau^2 / kappa0),
//   theta_s | mu, tau^2 ~ N(mu, tau^2),  sigma^2_s ~ Inv-chi^2(alpha0, sigma0^2),
//   x_sn ~ N(theta_s, sigma^2_s),
// with nu0 = 0.1, tau0^2 = 100, mu0 = 0, kappa0 = 0.1, alpha0 = 0.1, sigma0^2 = 10.  State
// (tau^2, mu, theta_1..S, sigma^2_1..S), D = 2 + 2S <= 32.  By conjugacy each update is a
// location-scale transform of its noise:
//   tau^2     = z_tau * A / (nu0 + S + 1),  A = nu0 tau0^2 + kappa0 (mu' - mu0)^2 + sum (theta'_s - mu')^2
//   mu        = (kappa0 mu0 + sum theta'_s) / (kappa0 + S) + sqrt(tau^2 / (kappa0 + S)) * n_mu
//   theta_s   = (mu / tau^2 + N xbar_s / sigma'^2_s) / P_s + n_s / sqrt(P_s),
//               P_s = 1 / tau^2 + N / sigma'^2_s
//   sigma^2_s = z_s * B_s / (alpha0 + N),  B_s = alpha0 sigma0^2 + sum_n (x_sn - theta_s)^2
// (primes: the previous sweep's values; z: Inv-chi^2(nu, 1) base variates, n: standard normals,
// all passed in as xi_t in the state's order).  sum_n (x_sn - theta)^2 is formed as the
// school's centred sum of squares plus N (xbar_s - theta)^2, so FP32 does not cancel.
//
// The Jacobian d f_t / d x_{t-1} is propagated forward through the updates: the rows of tau^2
// and mu are held per thread, each theta_s / sigma^2_s row follows from them and the unit
// direction of sigma'^2_s.  Dense rows are written as produced; the diagonal keeps two entries
// per school.  Gibbs has no accept step: every decision is 1 and the log-ratio 0.
#include "eval_small.cuh"

namespace pm {

namespace {

constexpr int kGibbsMaxS = 15;  // D = 2 + 2S <= 32

struct SchoolsModel {
    static constexpr double nu0 = 0.1, tau0sq = 100.0, mu0 = 0.0, kappa0 = 0.1, alpha0 = 0.1,
                            sigma0sq = 10.0;
};

// per-school mean and centred sum of squares of the scores (double accumulation)
template <typename R>
__device__ void school_stats(const R *X, int S, int N, R *xbar, R *ss) {
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        double m = 0.0;
        for (int n = 0; n < N; n++) m += (double)X[(size_t)k * N + n];
        m /= N;
        double q = 0.0;
        for (int n = 0; n < N; n++) {
            const double d = (double)X[(size_t)k * N + n] - m;
            q += d * d;
        }
        xbar[k] = (R)m;
        ss[k] = (R)q;
    }
}

// One sweep from sp with noise xi into out.  With jdense (D x D) or jd (D) the Jacobian (or its
// diagonal) is written, after damping and clip.
template <typename R>
__device__ void gibbs_sweep(int S, int N, const R *xbar, const R *ss, const R *sp, const R *xi,
                            R *out, R *jd, R *jdense, R damping, int clip) {
    using M = SchoolsModel;
    const int D = 2 + 2 * S;
    const bool want = jd || jdense;
    const R mu_p = sp[1];
    R A = (R)(M::nu0 * M::tau0sq) + (R)M::kappa0 * (mu_p - (R)M::mu0) * (mu_p - (R)M::mu0);
    R sum_dev = R(0), sum_th = R(0);
    for (int k = 0; k < S; k++) {
        const R dv = sp[2 + k] - mu_p;
        A += dv * dv;
        sum_dev += dv;
        sum_th += sp[2 + k];
    }
    const R nu_n = (R)M::nu0 + (R)(S + 1);
    const R tau2 = xi[0] * A / nu_n;
    const R kS = (R)M::kappa0 + (R)S;
    const R sd_mu = sqrt(tau2 / kS);
    const R mu = ((R)(M::kappa0 * M::mu0) + sum_th) / kS + sd_mu * xi[1];
    out[0] = tau2;
    out[1] = mu;
    // rows of tau^2 and mu over the previous state (tau^2' never enters: column 0 is zero)
    R dtau[32], dmu[32];
    if (want) {
        const R ct = xi[0] / nu_n;
#pragma unroll
        for (int j = 0; j < 32; j++) dtau[j] = R(0);
        dtau[1] = ct * (R(2) * (R)M::kappa0 * (mu_p - (R)M::mu0) - R(2) * sum_dev);
        for (int k = 0; k < S; k++) dtau[2 + k] = ct * R(2) * (sp[2 + k] - mu_p);
        const R c_mu = xi[1] / (R(2) * kS * sd_mu);  // d sd_mu / d tau^2
#pragma unroll
        for (int j = 0; j < 32; j++) dmu[j] = c_mu * dtau[j];
        for (int k = 0; k < S; k++) dmu[2 + k] += R(1) / kS;
        if (jdense) {
            for (int j = 0; j < D; j++) {
                jdense[j] = post_j(dtau[j], damping, clip);
                jdense[D + j] = post_j(dmu[j], damping, clip);
            }
        } else {
            jd[0] = post_j(dtau[0], damping, clip);
            jd[1] = post_j(dmu[1], damping, clip);
        }
    }
    const R an = (R)M::alpha0 + (R)N;
    const R itau2 = R(1) / tau2;
    for (int k = 0; k < S; k++) {
        const R sg = sp[2 + S + k];
        const R sx = (R)N * xbar[k];
        const R P = itau2 + (R)N / sg;
        const R a = mu * itau2 + sx / sg;
        const R sqP = sqrt(P);
        const R th = a / P + xi[2 + k] / sqP;
        const R dx = xbar[k] - th;
        const R B = (R)(M::alpha0 * M::sigma0sq) + ss[k] + (R)N * dx * dx;
        out[2 + k] = th;
        out[2 + S + k] = xi[2 + S + k] * B / an;
        if (!want) continue;
        const R c_sig = xi[2 + S + k] / an * (R(-2) * (R)N * dx);  // d sigma^2_s / d theta_s
        const R isg2 = R(1) / (sg * sg);
        // d theta along direction j of the previous state
        auto dth = [&](int j) -> R {
            R dP = -dtau[j] * itau2 * itau2;
            R da = dmu[j] * itau2 - mu * dtau[j] * itau2 * itau2;
            if (j == 2 + S + k) {
                dP -= (R)N * isg2;
                da -= sx * isg2;
            }
            return da / P - a * dP / (P * P) - R(0.5) * xi[2 + k] * dP / (P * sqP);
        };
        if (jdense) {
            R *rt = jdense + (size_t)(2 + k) * D, *rs = jdense + (size_t)(2 + S + k) * D;
            for (int j = 0; j < D; j++) {
                const R v = dth(j);
                rt[j] = post_j(v, damping, clip);
                rs[j] = post_j(c_sig * v, damping, clip);
            }
        } else {
            jd[2 + k] = post_j(dth(2 + k), damping, clip);
            jd[2 + S + k] = post_j(c_sig * dth(2 + S + k), damping, clip);
        }
    }
}

template <typename R, typename S_>
__global__ void __launch_bounds__(128) eval_gibbs_kernel(EvalArgs A) {
    if (A.skip && *(volatile const int *)A.skip) return;
    __shared__ R s_xbar[kGibbsMaxS], s_ss[kGibbsMaxS];
    const int D = A.D, S = (D - 2) / 2, N = A.N;
    school_stats<R>((const R *)A.X, S, N, s_xbar, s_ss);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double err = -INFINITY, rmax = 0.0;
    int acc_i = 1;
    if (t < A.T) {
        const R *s0 = (const R *)A.s0, *s = (const R *)A.s, *xin = (const R *)A.xi;
        const R *prev = t == 0 ? s0 : s + (size_t)(t - 1) * D;
        R sp[32], xi[32], f[32], jd[32];
        for (int d = 0; d < D; d++) {
            sp[d] = prev[d];
            xi[d] = xin[(size_t)t * D + d];
        }
        const int jac = A.jac;
        R *jdense = (jac == PMCMC_JAC_DENSE && A.a_out) ? (R *)A.a_out + (size_t)t * D * D : nullptr;
        const bool want_diag = jac == PMCMC_JAC_DIAG && A.a_out;
        gibbs_sweep<R>(S, N, s_xbar, s_ss, sp, xi, f, want_diag ? jd : nullptr, jdense,
                       (R)A.damping, A.clip);
        S_ *aout = (S_ *)A.a_out, *bout = (S_ *)A.b_out;
        R *fout = (R *)A.f_out;
        for (int d = 0; d < D; d++) {
            const R xc = s[(size_t)t * D + d];
            const R r = f[d] - xc;
            const double ar = fabs((double)r);
            const double e = ar - A.rtol * fabs((double)xc);
            err = isnan(e) ? INFINITY : max(err, e);
            rmax = isnan(ar) ? INFINITY : max(rmax, ar);
            if (bout) store_as<S_, R>(bout + (size_t)t * D + d, r);
            if (aout && jac != PMCMC_JAC_DENSE)
                store_as<S_, R>(aout + (size_t)t * D + d, want_diag ? jd[d] : R(0));
            if (fout) fout[(size_t)t * D + d] = f[d];
        }
        if (A.acc_out) A.acc_out[t] = 1;
        if (A.ell_out) A.ell_out[t] = 0.0;
    } else {
        acc_i = 0;
    }
    if (A.stats) reduce_stats(A.stats, err, rmax, (double)INFINITY, acc_i);
}

// the sequential chain: one thread walks t = 1..T
template <typename R>
__global__ void seq_gibbs_kernel(EvalArgs A) {
    __shared__ R s_xbar[kGibbsMaxS], s_ss[kGibbsMaxS];
    const int D = A.D, S = (D - 2) / 2, N = A.N;
    school_stats<R>((const R *)A.X, S, N, s_xbar, s_ss);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const R *xin = (const R *)A.xi;
    R *out = (R *)A.f_out;
    R x[32], xi[32], nx[32];
    for (int d = 0; d < D; d++) x[d] = ((const R *)A.s0)[d];
    for (int t = 0; t < A.T; t++) {
        for (int d = 0; d < D; d++) xi[d] = xin[(size_t)t * D + d];
        gibbs_sweep<R>(S, N, s_xbar, s_ss, x, xi, nx, nullptr, nullptr, R(1), 0);
        for (int d = 0; d < D; d++) {
            x[d] = nx[d];
            out[(size_t)t * D + d] = nx[d];
        }
        if (A.acc_out) A.acc_out[t] = 1;
    }
}

}  // namespace

bool gibbs_supported(int D, int N) { return D >= 4 && D % 2 == 0 && (D - 2) / 2 <= kGibbsMaxS && N >= 1; }

template <typename R, typename S_>
cudaError_t launch_gibbs(const EvalArgs &A, cudaStream_t st, bool seq) {
    if (!gibbs_supported(A.D, A.N)) return cudaErrorInvalidValue;
    if (seq) {
        seq_gibbs_kernel<R><<<1, 32, 0, st>>>(A);
    } else {
        eval_gibbs_kernel<R, S_><<<ceil_div(A.T, 128), 128, 0, st>>>(A);
    }
    return cudaGetLastError();
}

template cudaError_t launch_gibbs<float, float>(const EvalArgs &, cudaStream_t, bool);
template cudaError_t launch_gibbs<double, double>(const EvalArgs &, cudaStream_t, bool);
template cudaError_t launch_gibbs<float, __nv_bfloat16>(const EvalArgs &, cudaStream_t, bool);

}  // namespace pm
