// Evaluate-and-linearise pass for Bayesian logistic regression (the target of Section 5.2):
//   log p(x) = sum_n [y_n z_n - log(1 + e^{z_n})] - |x|^2 / (2 sigma_p^2),   z = X x,
//   grad = X^T (y - sigmoid(z)) - x / sigma_p^2,
//   H v  = -X^T (w (.) X v) - v / sigma_p^2,  w = sigmoid(z)(1 - sigmoid(z)).
//
// Each CTA owns TT consecutive timesteps.  Every gradient or Hessian-vector product over its
// TT states is a pair of dense contractions with the shared design matrix,
//   Z = V X^T  (TT x N),   elementwise map,   G = C X  (TT x D),
// so a CTA streams X through shared memory in sub-chunks of NC rows and reuses each X row for
// all TT states.  All per-timestep vectors stay in shared memory; HBM traffic is the states,
// the noise and the outputs.  The MH log-ratio is accumulated in FP64 (per-thread FP32 partial
// sums of at most NC/16 terms, reduced in FP64).
//
// Passes of one MALA linearisation (Section 3.2):
//   1. grad at x (+ sum of log-likelihood terms, + diag(X^T W X) for the exact diagonal)
//   2. grad at x~ (+ log-likelihood sum)             -> ell, decision, e = x - x~ - eps g(x~)
//   3. H(x~) e,   4. H(x) v  (only when some step of the tile has an active gate term)
// For the dense Jacobian the per-(t, n) weights w(x) are written out and a separate kernel
// assembles J_t = g (I + eps H(x)) + (1 - g) I + u_t v_t^T.
#include "common.cuh"
#include "eval.h"
#include "seq.h"
#include "logreg_tile.cuh"

namespace pm {

using namespace lr;

template <typename R, typename S_, int DP>
__global__ void __launch_bounds__(kNT) eval_logreg_kernel(EvalArgs A) {
    if (A.skip && *(volatile const int *)A.skip) return;
    using G = Geo<DP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R, DP> &S = *reinterpret_cast<Smem<R, DP> *>(smem_raw);
    constexpr int TT = G::TT;
    const int T = A.T, D = A.D, N = A.N;
    const int t0 = blockIdx.x * TT;
    const int tid = threadIdx.x;
    const R eps = (R)A.eps, sp2 = (R)(A.sigma_p * A.sigma_p), inv_sp2 = R(1) / sp2;
    const R *s0 = (const R *)A.s0, *s = (const R *)A.s, *xin = (const R *)A.xi;
    const R *Xp = (const R *)A.Xp, *y = (const R *)A.y;
    const int jac = A.jac;
    const bool want_gate = A.gate_grad && jac != PMCMC_JAC_ZERO;
    const bool want_dh = jac == PMCMC_JAC_DIAG;

    // load the states s_{t-1}, s_t and the noise of this tile (zero padded to DP)
    for (int e = tid; e < TT * DP; e += kNT) {
        const int tl = e / DP, d = e - tl * DP;
        const int t = t0 + tl;
        R xp = R(0), xv = R(0), sv = R(0);
        if (t < T && d < D) {
            xp = t == 0 ? s0[d] : s[(size_t)(t - 1) * D + d];
            xv = xin[(size_t)t * D + d];
            sv = s[(size_t)t * D + d];
        }
        S.x[e] = xp;
        S.xi[e] = xv;
        S.sc[e] = sv;
        S.dh[e] = R(0);
    }
    if (tid < TT) S.ll[tid] = 0.0;
    __syncthreads();

    // pass 1: gradient at x
    xpass<R, DP, kGrad>(S, Xp, y, N, S.x, nullptr, S.g, true, want_dh,
                        jac == PMCMC_JAC_DENSE ? (R *)A.w_out : nullptr, t0, T);
    double *llx = S.ell;  // reuse as scratch for log-lik at x
    if (tid < TT) {
        llx[tid] = S.ll[tid];
        S.ll[tid] = 0.0;
    }
    const R sq = sqrt(R(2) * eps);
    for (int e = tid; e < TT * DP; e += kNT) {
        S.g[e] -= S.x[e] * inv_sp2;
        S.xt[e] = S.x[e] + eps * S.g[e] + sq * S.xi[e];
    }
    __syncthreads();
    // pass 2: gradient at x~
    xpass<R, DP, kGrad>(S, Xp, y, N, S.xt, nullptr, S.gt, true, false, nullptr, t0, T);
    for (int e = tid; e < TT * DP; e += kNT) {
        S.gt[e] -= S.xt[e] * inv_sp2;
        S.e[e] = S.x[e] - S.xt[e] - eps * S.gt[e];
    }
    __syncthreads();
    // ell = [ll(x~) - |x~|^2/2sp2] - [ll(x) - |x|^2/2sp2] - |e|^2/(4 eps) + |xi|^2/2
    per_t_sum<R, DP>(TT, [&](int t, int d) {
        const int k = t * DP + d;
        const double xt = S.xt[k], x = S.x[k], e = S.e[k], xi = S.xi[k];
        return -(xt * xt - x * x) / (2.0 * (double)sp2) - e * e / (4.0 * (double)eps) + 0.5 * xi * xi;
    }, S.gtl);
    __syncthreads();
    int any_gate = 0;
    if (tid < TT) {
        const double ell = (S.ll[tid] - llx[tid]) + S.gtl[tid];
        const int t = t0 + tid;
        const double u = t < T ? A.u[t] : 0.5;
        const double la = (ell < 0.0 || isnan(ell)) ? ell : 0.0;
        const double gtl = la - log(u);
        S.acc[tid] = (t < T) && gtl > 0.0;
        S.cg[tid] = R(0);
        if (want_gate && ell < 0.0 && t < T) {
            const double sg = 1.0 / (1.0 + exp(-gtl));
            S.cg[tid] = (R)(sg * (1.0 - sg));
            any_gate = 1;
        }
        if (A.ell_out && t < T) A.ell_out[t] = ell;
        if (A.acc_out && t < T) A.acc_out[t] = S.acc[tid] ? 1 : 0;
        S.ll[tid] = ell;  // keep ell
        S.gtl[tid] = gtl;
    }
    any_gate = __syncthreads_or(any_gate);

    if (any_gate) {
        // pass 3: H(x~) e
        xpass<R, DP, kHvp>(S, Xp, y, N, S.xt, S.e, S.v, false, false, nullptr, t0, T);
        const R inv2e = R(1) / (R(2) * eps);
        for (int e = tid; e < TT * DP; e += kNT) {
            const R He = -S.v[e] - S.e[e] * inv_sp2;
            S.v[e] = S.gt[e] + (S.e[e] + eps * He) * inv2e;
        }
        __syncthreads();
        // pass 4: H(x) v
        xpass<R, DP, kHvp>(S, Xp, y, N, S.x, S.v, S.gl, false, false, nullptr, t0, T);
        for (int e = tid; e < TT * DP; e += kNT) {
            const R Hv = -S.gl[e] - S.v[e] * inv_sp2;
            S.gl[e] = S.v[e] + eps * Hv - S.g[e] - S.e[e] * inv2e;
        }
        __syncthreads();
    } else {
        for (int e = tid; e < TT * DP; e += kNT) S.gl[e] = R(0);
        __syncthreads();
    }
    // Hutchinson probe: H(x) z
    if (jac == PMCMC_JAC_DIAG_HUTCH) {
        const int it = A.iter ? *A.iter : 0;
        for (int e = tid; e < TT * DP; e += kNT) {
            const int tl = e / DP, d = e - tl * DP;
            R z = R(0);
            if (d < D && t0 + tl < T) {
                uint4 w = philox4x32_10(make_uint4((unsigned)(d >> 7), (unsigned)(t0 + tl), A.chain, 2u + (unsigned)it),
                                        make_uint2((unsigned)A.seed, (unsigned)(A.seed >> 32)));
                const int dd = d & 127;
                unsigned int word = dd < 32 ? w.x : (dd < 64 ? w.y : (dd < 96 ? w.z : w.w));
                z = ((word >> (dd & 31)) & 1u) ? R(1) : R(-1);
            }
            S.e[e] = z;  // e is no longer needed
        }
        __syncthreads();
        xpass<R, DP, kHvp>(S, Xp, y, N, S.x, S.e, S.v, false, false, nullptr, t0, T);
        per_t_sum<R, DP>(TT, [&](int t, int d) { return (double)S.gl[t * DP + d] * (double)S.e[t * DP + d]; }, S.ell);
        __syncthreads();
    }

    // outputs: f, r = f - s_t, J
    const R damping = (R)A.damping;
    double err = -INFINITY, rmax = 0.0;
    S_ *aout = (S_ *)A.a_out, *bout = (S_ *)A.b_out;
    R *fout = (R *)A.f_out;
    R *ru = (R *)A.rank1_u, *rv = (R *)A.rank1_v;
    for (int e = tid; e < TT * DP; e += kNT) {
        const int tl = e / DP, d = e - tl * DP;
        const int t = t0 + tl;
        if (t >= T || d >= D) continue;
        const bool acc = S.acc[tl];
        const R f = acc ? S.xt[e] : S.x[e];
        const R r = f - S.sc[e];
        const double ar = fabs((double)r);
        const double ee = ar - A.rtol * fabs((double)S.sc[e]);
        err = isnan(ee) ? INFINITY : max(err, ee);
        rmax = isnan(ar) ? INFINITY : max(rmax, ar);
        const size_t o = (size_t)t * D + d;
        if (bout) store_as<S_, R>(bout + o, r);
        if (fout) fout[o] = f;
        const R ga = acc ? R(1) : R(0);
        const R gterm = S.cg[tl] * (S.xt[e] - S.x[e]);
        if (jac == PMCMC_JAC_DIAG) {
            const R Hdd = -S.dh[e] - inv_sp2;
            const R j = ga * (R(1) + eps * Hdd) + (R(1) - ga) + gterm * S.gl[e];
            if (aout) store_as<S_, R>(aout + o, post_j(j, damping, A.clip));
        } else if (jac == PMCMC_JAC_DIAG_HUTCH) {
            const R z = S.e[e];
            const R Hz = -S.v[e] - z * inv_sp2;
            const R j = z * (z + ga * eps * Hz + gterm * (R)S.ell[tl]);
            if (aout) store_as<S_, R>(aout + o, post_j(j, damping, A.clip));
        } else if (jac == PMCMC_JAC_ZERO) {
            if (aout) store_as<S_, R>(aout + o, R(0));
        } else {  // dense: rank-one gate term for the assembly kernel
            if (ru) ru[o] = gterm;
            if (rv) rv[o] = S.gl[e];
        }
    }
    double margin = INFINITY;
    int acc_i = 0;
    if (tid < TT && t0 + tid < T) {
        margin = fabs(S.gtl[tid]);
        acc_i = S.acc[tid];
    }
    if (A.stats) {
        // block reduction
        __shared__ double red[4][kNT / 32];
        const int lane = tid & 31, w = tid >> 5;
        double e1 = warp_max(err), e2 = warp_max(rmax), e3 = warp_min(margin);
        double e4 = warp_sum((double)acc_i);
        if (lane == 0) {
            red[0][w] = e1;
            red[1][w] = e2;
            red[2][w] = e3;
            red[3][w] = e4;
        }
        __syncthreads();
        if (w == 0) {
            e1 = lane < kNT / 32 ? red[0][lane] : -INFINITY;
            e2 = lane < kNT / 32 ? red[1][lane] : 0.0;
            e3 = lane < kNT / 32 ? red[2][lane] : INFINITY;
            e4 = lane < kNT / 32 ? red[3][lane] : 0.0;
            e1 = warp_max(e1);
            e2 = warp_max(e2);
            e3 = warp_min(e3);
            e4 = warp_sum(e4);
            if (lane == 0) {
                atomic_max_d(&A.stats->err, e1);
                atomic_max_d(&A.stats->rmax, e2);
                atomic_min_d(&A.stats->min_margin, e3);
                if (e4 > 0) atomicAdd(&A.stats->accepts, (unsigned long long)(e4 + 0.5));
            }
        }
    }
}

// ==========================================================================================
// Dense Jacobian assembly for logistic MALA (DEER, Eq. 2):
//   J_t = g_t (I + eps H_t) + (1 - g_t) I + u_t v_t^T,   H_t = -sum_n w_tn X_n X_n^T - I/sp^2.
// One CTA per 8 timesteps; thread owns (d1, d2) pairs for all 8 timesteps.
// ==========================================================================================
template <typename R, int DP>
__global__ void __launch_bounds__(256) logreg_dense_jac_kernel(EvalArgs A) {
    if (A.skip && *(volatile const int *)A.skip) return;
    constexpr int TB = 8, NB = 32;
    __shared__ R Xs[NB][DP];
    __shared__ R Wsh[TB][NB];
    const int T = A.T, D = A.D, N = A.N, DD = D * D;
    const int t0 = blockIdx.x * TB;
    const R *Xp = (const R *)A.Xp, *W = (const R *)A.w_out;
    constexpr int PMAX = (DP * DP + 255) / 256;
    R acc[PMAX][TB];
#pragma unroll
    for (int p = 0; p < PMAX; p++)
#pragma unroll
        for (int i = 0; i < TB; i++) acc[p][i] = R(0);
    for (int n0 = 0; n0 < N; n0 += NB) {
        __syncthreads();
        for (int e = threadIdx.x; e < NB * DP; e += 256) {
            const int r = e / DP, k = e % DP;
            Xs[r][k] = Xp[(size_t)(n0 + r) * DP + k];
        }
        for (int e = threadIdx.x; e < TB * NB; e += 256) {
            const int i = e / NB, r = e % NB;
            Wsh[i][r] = (t0 + i < T && n0 + r < N) ? W[(size_t)(t0 + i) * N + n0 + r] : R(0);
        }
        __syncthreads();
        for (int r = 0; r < NB; r++) {
#pragma unroll
            for (int p = 0; p < PMAX; p++) {
                const int q = threadIdx.x + 256 * p;
                if (q < DD) {
                    const int d1 = q / D, d2 = q - d1 * D;
                    const R xx = Xs[r][d1] * Xs[r][d2];
#pragma unroll
                    for (int i = 0; i < TB; i++) acc[p][i] = fma(Wsh[i][r], xx, acc[p][i]);
                }
            }
        }
    }
    const R eps = (R)A.eps, inv_sp2 = R(1) / (R)(A.sigma_p * A.sigma_p), damping = (R)A.damping;
    const R *ru = (const R *)A.rank1_u, *rv = (const R *)A.rank1_v;
    R *J = (R *)A.a_out;
#pragma unroll
    for (int p = 0; p < PMAX; p++) {
        const int q = threadIdx.x + 256 * p;
        if (q >= DD) continue;
        const int d1 = q / D, d2 = q - d1 * D;
#pragma unroll
        for (int i = 0; i < TB; i++) {
            const int t = t0 + i;
            if (t >= T) continue;
            const R ga = A.acc_out[t] ? R(1) : R(0);
            const R H = -acc[p][i] - (d1 == d2 ? inv_sp2 : R(0));
            R v = ga * eps * H + (d1 == d2 ? R(1) : R(0)) + ru[(size_t)t * D + d1] * rv[(size_t)t * D + d2];
            J[(size_t)t * DD + q] = post_j(v, damping, A.clip);
        }
    }
}

// ==========================================================================================
// Sequential logistic MALA / HMC on the GPU: one CTA walks t = 1..T; each gradient is a block
// reduction over the rows of X.  This is the paper's sequential baseline on the same device.
// ==========================================================================================
template <typename R>
__device__ R block_sum(R v, R *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    R s = R(0);
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    return s;
}

// Gradient at x (into g, shared) and the log-likelihood sum.  Rows are spread over the
// threads for z_n = X_n . x; the reduction over rows is split into P = blockDim / D row classes
// per coordinate and summed in shared memory (no atomics).
template <typename R>
__device__ double seq_grad(const R *__restrict__ X, const R *__restrict__ y, int N, int D,
                           const R *x, R *g, R *cbuf, R *part, R inv_sp2, double *red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double ll = 0.0;
    for (int n = tid; n < N; n += nt) {
        const R *Xn = X + (size_t)n * D;
        R z = R(0);
        for (int d = 0; d < D; d++) z = fma(Xn[d], x[d], z);
        cbuf[n] = y[n] - sigm(z);
        ll += (double)(y[n] * z - softplus(z));
    }
    ll = warp_sum(ll);
    if ((tid & 31) == 0) red[tid >> 5] = ll;
    __syncthreads();
    const int P = max(1, nt / D);
    if (tid < P * D) {
        const int d = tid % D, pc = tid / D;
        R acc = R(0);
        for (int n = pc; n < N; n += P) acc = fma(cbuf[n], X[(size_t)n * D + d], acc);
        part[pc * D + d] = acc;
    }
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nt / 32; i++) s += red[i];
    for (int d = tid; d < D; d += nt) {
        R acc = R(0);
        for (int pc = 0; pc < P; pc++) acc += part[pc * D + d];
        g[d] = acc - x[d] * inv_sp2;
    }
    __syncthreads();
    return s;
}

template <typename R>
__global__ void __launch_bounds__(256) seq_logreg_kernel(EvalArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = A.D, N = A.N, L = A.L;
    R *x = (R *)smem_raw;
    R *xt = x + D, *g = xt + D, *gt = g + D, *v = gt + D;
    R *cbuf = v + D, *part = cbuf + N;  // N row weights, blockDim partial sums
    __shared__ double red[32];
    const R *X = (const R *)A.X, *y = (const R *)A.y, *xin = (const R *)A.xi;
    R *out = (R *)A.f_out;
    const R eps = (R)A.eps, inv_sp2 = R(1) / (R)(A.sigma_p * A.sigma_p);
    const int tid = threadIdx.x;
    for (int d = tid; d < D; d += blockDim.x) x[d] = ((const R *)A.s0)[d];
    __syncthreads();
    for (int t = 0; t < A.T; t++) {
        const R *xi = xin + (size_t)t * D;
        bool acc;
        if (A.sampler == PMCMC_MALA) {
            double llx = seq_grad<R>(X, y, N, D, x, g, cbuf, part, inv_sp2, red);
            const R sq = sqrt(R(2) * eps);
            for (int d = tid; d < D; d += blockDim.x) xt[d] = x[d] + eps * g[d] + sq * xi[d];
            __syncthreads();
            double llt = seq_grad<R>(X, y, N, D, xt, gt, cbuf, part, inv_sp2, red);
            double part = 0.0;
            for (int d = tid; d < D; d += blockDim.x) {
                const double e = (double)x[d] - (double)xt[d] - (double)eps * (double)gt[d];
                part += -((double)xt[d] * xt[d] - (double)x[d] * x[d]) * 0.5 * (double)inv_sp2 -
                        e * e / (4.0 * (double)eps) + 0.5 * (double)xi[d] * xi[d];
            }
            part = warp_sum(part);
            __syncthreads();
            if ((tid & 31) == 0) red[tid >> 5] = part;
            __syncthreads();
            double q = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); i++) q += red[i];
            const double ell = llt - llx + q;
            const double la = (ell < 0.0 || isnan(ell)) ? ell : 0.0;
            acc = la - log(A.u[t]) > 0.0;
            __syncthreads();
            if (acc)
                for (int d = tid; d < D; d += blockDim.x) x[d] = xt[d];
        } else {
            // HMC: v0 = xi, half step, L leapfrogs, negative half step
            double ll0 = seq_grad<R>(X, y, N, D, x, g, cbuf, part, inv_sp2, red);
            double pe = 0.0;
            for (int d = tid; d < D; d += blockDim.x) {
                pe += 0.5 * (double)xi[d] * xi[d] + 0.5 * (double)inv_sp2 * (double)x[d] * x[d];
                xt[d] = x[d];
                v[d] = xi[d] + R(0.5) * eps * g[d];
            }
            double H0 = block_sum<double>(pe, red) - ll0;
            __syncthreads();
            double llL = ll0;
            for (int k = 0; k < L; k++) {
                for (int d = tid; d < D; d += blockDim.x) xt[d] += eps * v[d];
                __syncthreads();
                llL = seq_grad<R>(X, y, N, D, xt, gt, cbuf, part, inv_sp2, red);
                for (int d = tid; d < D; d += blockDim.x) v[d] += eps * gt[d];
                __syncthreads();
            }
            pe = 0.0;
            for (int d = tid; d < D; d += blockDim.x) {
                const R gl = L > 0 ? gt[d] : g[d];
                v[d] -= R(0.5) * eps * gl;
                pe += 0.5 * (double)v[d] * v[d] + 0.5 * (double)inv_sp2 * (double)xt[d] * xt[d];
            }
            double HL = block_sum<double>(pe, red) - llL;
            const double diff = H0 - HL;
            const double la = (diff < 0.0 || isnan(diff)) ? diff : 0.0;
            acc = la - log(A.u[t]) > 0.0;
            __syncthreads();
            if (acc)
                for (int d = tid; d < D; d += blockDim.x) x[d] = xt[d];
        }
        __syncthreads();
        for (int d = tid; d < D; d += blockDim.x) out[(size_t)t * D + d] = x[d];
        if (tid == 0 && A.acc_out) A.acc_out[t] = acc ? 1 : 0;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
int logreg_padded_dim(int D) {
    if (D <= 16) return 16;
    if (D <= 32) return 32;
    if (D <= 64) return 64;
    if (D <= 128) return 128;
    return -1;
}

template <typename R, typename S_, int DP>
static cudaError_t run_eval_logreg(const EvalArgs &A, cudaStream_t st) {
    const size_t sm = sizeof(Smem<R, DP>);
    auto k = eval_logreg_kernel<R, S_, DP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<ceil_div(A.T, Geo<DP>::TT), kNT, sm, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_eval_logreg(const EvalArgs &A, cudaStream_t st) {
    if (A.tc_img && logreg_tc_supported(A)) return launch_eval_logreg_tc(A, st);
    const int DP = logreg_padded_dim(A.D);
#define PM_LR(R_, S_)                                                   \
    switch (DP) {                                                       \
    case 16: return run_eval_logreg<R_, S_, 16>(A, st);                 \
    case 32: return run_eval_logreg<R_, S_, 32>(A, st);                 \
    case 64: return run_eval_logreg<R_, S_, 64>(A, st);                 \
    case 128: return run_eval_logreg<R_, S_, 128>(A, st);               \
    default: return cudaErrorInvalidValue;                              \
    }
    if (A.f64) {
        if (DP > 64) return cudaErrorInvalidValue;
        switch (DP) {
        case 16: return run_eval_logreg<double, double, 16>(A, st);
        case 32: return run_eval_logreg<double, double, 32>(A, st);
        case 64: return run_eval_logreg<double, double, 64>(A, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (A.bf16) PM_LR(float, __nv_bfloat16)
    PM_LR(float, float)
#undef PM_LR
}

cudaError_t launch_logreg_dense_jac(const EvalArgs &A, cudaStream_t st) {
    if (A.pair_img && !A.f64) return launch_jac_logreg_tc(A, st);
    const int DP = logreg_padded_dim(A.D);
    const int blocks = ceil_div(A.T, 8);
#define PM_DJ(R_)                                                                             \
    switch (DP) {                                                                             \
    case 16: logreg_dense_jac_kernel<R_, 16><<<blocks, 256, 0, st>>>(A); break;               \
    case 32: logreg_dense_jac_kernel<R_, 32><<<blocks, 256, 0, st>>>(A); break;               \
    default: return cudaErrorInvalidValue;                                                    \
    }
    if (A.f64) {
        PM_DJ(double)
    } else {
        PM_DJ(float)
    }
#undef PM_DJ
    return cudaGetLastError();
}

cudaError_t launch_seq_logreg(const EvalArgs &A, cudaStream_t st) {
    {
        SeqChain ch = seq_chain_from(A);
        if (seq_fast_supported(ch) && seq_cluster_size(ch, A.f64) > 0) return launch_seq_chain(ch, A.f64, st);
    }
    // fallback for designs too large for the shared memory of a 16-CTA cluster: one CTA that
    // reads the design from global memory
    const size_t sm = (A.f64 ? 8 : 4) * ((size_t)5 * A.D + A.N + 256);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    if (A.f64)
        cudaFuncSetAttribute(seq_logreg_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else
        cudaFuncSetAttribute(seq_logreg_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (A.f64)
        seq_logreg_kernel<double><<<1, 256, sm, st>>>(A);
    else
        seq_logreg_kernel<float><<<1, 256, sm, st>>>(A);
    return cudaGetLastError();
}

}  // namespace pm
