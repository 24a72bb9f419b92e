// HMC with the leapfrog integration itself solved in parallel (Section 3.3, Algorithm 2).
// The HMC steps t = 1..T run one after another; inside each step the L leapfrog updates
//   s_k = f(s_{k-1}) = [x + eps v,  v + eps grad log p(x + eps v)],   k = 1..L   (Eq. 7)
// from s_0 = [x_0, v_0 + eps/2 grad log p(x_0)] are the fixed point solved by block
// quasi-DEER: the Jacobian of Eq. 8 keeps the diagonal of each D x D block,
//   J_k = [[I, eps I], [eps diag H(x'), I + eps^2 diag H(x')]],  x' = x_{k-1} + eps v_{k-1},
// and the linear recursion over 2x2-block-diagonal maps is a scan whose combine is the
// 8-elementwise-product rule of Appendix A.3.  One warp per chain: lane k owns leapfrog step
// k+1, the scan is a warp-shuffle Hillis-Steele scan, and the residual check a warp max.
#include "common.cuh"
#include "solve.h"
#include "targets.cuh"

namespace pm {

namespace {

template <typename R>
__device__ __forceinline__ R post_j(R v, R damping, int clip) {
    v *= damping;
    if (clip) v = v > R(1) ? R(1) : (v < R(-1) ? R(-1) : v);
    return v;
}

template <typename R, int DM, class TG>
__device__ __forceinline__ R diag_hess(const TG &tg, const R *x, int d) {
    return tg.hess(x, d, d);
}

}  // namespace

template <typename R, int DM, int TGT>
__global__ void __launch_bounds__(32) par_leapfrog_kernel(EvalArgs A, int max_inner,
                                                          double atol, CtlBlock *ctl) {
    __shared__ R smu[DM];
    __shared__ R sP[DM * DM];
    const int D = A.D, L = A.L, lane = threadIdx.x;
    if (TGT == PMCMC_GAUSSIAN) {
        const R *mu = (const R *)A.mu, *P = (const R *)A.P;
        for (int e = lane; e < DM * DM; e += 32) {
            const int i = e / DM, j = e % DM;
            sP[e] = (i < D && j < D) ? P[i * D + j] : R(0);
        }
        for (int d = lane; d < DM; d += 32) smu[d] = d < D ? mu[d] : R(0);
        __syncwarp();
    }
    using TG = typename std::conditional<TGT == PMCMC_GAUSSIAN, GaussianT<R, DM>,
                                         BananaT<R, (DM == 2 ? 2 : 2)>>::type;
    TG tg;
    if constexpr (TGT == PMCMC_GAUSSIAN) {
        tg.mu = smu;
        tg.P = sP;
    }
    const R eps = (R)A.eps, he = R(0.5) * eps, damping = (R)A.damping;
    const R *xin = (const R *)A.xi;
    R *out = (R *)A.f_out;
    const bool active = lane < L;
    R x0[DM], g0[DM];
#pragma unroll
    for (int d = 0; d < DM; d++) x0[d] = d < D ? ((const R *)A.s0)[d] : R(0);
    unsigned long long total_inner = 0, max_inner_seen = 0;
    unsigned long long accepts = 0;
    double min_margin = INFINITY;
    for (int t = 0; t < A.T; t++) {
        R xi[DM];
#pragma unroll
        for (int d = 0; d < DM; d++) xi[d] = d < D ? xin[(size_t)t * D + d] : R(0);
        tg.grad(x0, g0);
        double vv = 0.0;
#pragma unroll
        for (int d = 0; d < DM; d++) vv += (double)xi[d] * (double)xi[d];
        const double H0 = 0.5 * vv - tg.logp(x0, g0);
        // inner initial state s_0 and guess s_k = s_0
        R sx0[DM], sv0[DM], sx[DM], sv[DM];
#pragma unroll
        for (int d = 0; d < DM; d++) {
            sx0[d] = x0[d];
            sv0[d] = xi[d] + he * g0[d];
            sx[d] = sx0[d];
            sv[d] = sv0[d];
        }
        int it = 0;
        for (;;) {
            // previous state of lane k is lane k-1's state (lane 0: s_0)
            R px[DM], pv[DM];
#pragma unroll
            for (int d = 0; d < DM; d++) {
                R ux = __shfl_up_sync(0xffffffffu, sx[d], 1);
                R uv = __shfl_up_sync(0xffffffffu, sv[d], 1);
                px[d] = lane == 0 ? sx0[d] : ux;
                pv[d] = lane == 0 ? sv0[d] : uv;
            }
            // f(prev) and the block Jacobian at prev
            R fx[DM], fv[DM], g[DM];
#pragma unroll
            for (int d = 0; d < DM; d++) fx[d] = px[d] + eps * pv[d];
            tg.grad(fx, g);
            R ja[DM], jb[DM], jc[DM], jd[DM], rx[DM], rv[DM];
            double err = -INFINITY;
#pragma unroll
            for (int d = 0; d < DM; d++) {
                fv[d] = pv[d] + eps * g[d];
                const R h = diag_hess<R, DM>(tg, fx, d);
                ja[d] = post_j(R(1), damping, A.clip);
                jb[d] = post_j(eps, damping, A.clip);
                jc[d] = post_j(eps * h, damping, A.clip);
                jd[d] = post_j(R(1) + eps * eps * h, damping, A.clip);
                rx[d] = fx[d] - sx[d];
                rv[d] = fv[d] - sv[d];
                if (active && d < D) {
                    double e1 = fabs((double)rx[d]) - A.rtol * fabs((double)sx[d]);
                    double e2 = fabs((double)rv[d]) - A.rtol * fabs((double)sv[d]);
                    e1 = isnan(e1) ? INFINITY : e1;
                    e2 = isnan(e2) ? INFINITY : e2;
                    err = max(err, max(e1, e2));
                }
            }
            err = warp_max(err);
            if (err <= atol || it >= max_inner) break;
            if (!active) {
#pragma unroll
                for (int d = 0; d < DM; d++) {
                    ja[d] = jd[d] = R(1);
                    jb[d] = jc[d] = R(0);
                    rx[d] = rv[d] = R(0);
                }
            }
            // inclusive warp scan of the block maps (Appendix A.3 combine)
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int d = 0; d < DM; d++) {
                    const R pa = __shfl_up_sync(0xffffffffu, ja[d], off);
                    const R pb = __shfl_up_sync(0xffffffffu, jb[d], off);
                    const R pc = __shfl_up_sync(0xffffffffu, jc[d], off);
                    const R pd = __shfl_up_sync(0xffffffffu, jd[d], off);
                    const R prx = __shfl_up_sync(0xffffffffu, rx[d], off);
                    const R prv = __shfl_up_sync(0xffffffffu, rv[d], off);
                    if (lane >= off) {
                        // (M, r) o (M', r') = (M M', M r' + r)
                        const R na = ja[d] * pa + jb[d] * pc;
                        const R nb = ja[d] * pb + jb[d] * pd;
                        const R nc = jc[d] * pa + jd[d] * pc;
                        const R nd = jc[d] * pb + jd[d] * pd;
                        const R nrx = ja[d] * prx + jb[d] * prv + rx[d];
                        const R nrv = jc[d] * prx + jd[d] * prv + rv[d];
                        ja[d] = na;
                        jb[d] = nb;
                        jc[d] = nc;
                        jd[d] = nd;
                        rx[d] = nrx;
                        rv[d] = nrv;
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < DM; d++) {
                R nx = sx[d] + rx[d], nv = sv[d] + rv[d];
                if (!isfinite(nx) || !isfinite(nv)) {
                    nx = sx0[d];
                    nv = sv0[d];
                }
                sx[d] = nx;
                sv[d] = nv;
            }
            it++;
        }
        total_inner += it;
        max_inner_seen = max(max_inner_seen, (unsigned long long)it);
        // x_L, v_L from the last leapfrog step; negative half step; energy; accept
        R xL[DM], vL[DM], gL[DM];
#pragma unroll
        for (int d = 0; d < DM; d++) {
            xL[d] = __shfl_sync(0xffffffffu, sx[d], L - 1);
            vL[d] = __shfl_sync(0xffffffffu, sv[d], L - 1);
        }
        tg.grad(xL, gL);
        vv = 0.0;
#pragma unroll
        for (int d = 0; d < DM; d++) {
            vL[d] -= he * gL[d];
            vv += (double)vL[d] * (double)vL[d];
        }
        const double HL = 0.5 * vv - tg.logp(xL, gL);
        const double diff = H0 - HL;
        const double la = (diff < 0.0 || isnan(diff)) ? diff : 0.0;
        const double gtl = la - log(A.u[t]);
        const bool acc = gtl > 0.0;
        min_margin = min(min_margin, fabs(gtl));
        accepts += acc;
        if (acc) {
#pragma unroll
            for (int d = 0; d < DM; d++) x0[d] = xL[d];
        }
        if (lane == 0) {
            for (int d = 0; d < D; d++) out[(size_t)t * D + d] = x0[d];
            if (A.acc_out) A.acc_out[t] = acc ? 1 : 0;
        }
    }
    if (lane == 0) {
        ctl->inner_iters = total_inner;
        ctl->inner_max = max_inner_seen;
        ctl->stats[0].accepts = accepts;
        ctl->stats[0].min_margin = ord_encode(min_margin);
    }
}

pmcmc_status solve_par_leapfrog(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o,
                                int T, const void *s0, const void *xi, const double *u,
                                void *s_out, pmcmc_result *res, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int D = tg->D;
    if (o->leapfrog_L > 32) return set_error(c, PMCMC_EUNSUPPORTED, "parallel leapfrog supports L <= 32");
    if (tg->kind == PMCMC_LOGREG)
        return set_error(c, PMCMC_EUNSUPPORTED, "parallel leapfrog supports Gaussian and banana targets");
    if (o->jac != PMCMC_JAC_BLOCK2)
        return set_error(c, PMCMC_EINVAL, "parallel leapfrog uses the BLOCK2 Jacobian");
    const bool f64 = o->precision == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    void *gxi = nullptr;
    double *gu = nullptr;
    if (!xi) {
        Carve cv;
        size_t ox = cv.take((size_t)rb * T * D), ou = cv.take(sizeof(double) * T);
        pmcmc_status ps = ws_reserve(c, cv.used);
        if (ps != PMCMC_OK) return ps;
        gxi = (char *)c->ws + ox;
        gu = (double *)((char *)c->ws + ou);
        cudaError_t e = launch_noise(o->seed, o->chain_id, T, D, f64, gxi, gu, st);
        if (e != cudaSuccess) return set_error(c, PMCMC_ECUDA, cudaGetErrorString(e));
        xi = gxi;
        u = gu;
    }
    EvalArgs A;
    fill_eval_args(A, tg, o, T);
    A.s0 = s0;
    A.xi = xi;
    A.u = u;
    A.f_out = s_out;
    const int max_inner = o->max_iters > 0 ? o->max_iters : o->leapfrog_L;
    cudaEventRecord(c->ev0, st);
#define PM_PL(R_, DM_, TGT_) par_leapfrog_kernel<R_, DM_, TGT_><<<1, 32, 0, st>>>(A, max_inner, o->atol, c->ctl)
    if (tg->kind == PMCMC_BANANA) {
        if (f64) PM_PL(double, 2, PMCMC_BANANA); else PM_PL(float, 2, PMCMC_BANANA);
    } else {
        if (D <= 2) { if (f64) PM_PL(double, 2, PMCMC_GAUSSIAN); else PM_PL(float, 2, PMCMC_GAUSSIAN); }
        else if (D <= 4) { if (f64) PM_PL(double, 4, PMCMC_GAUSSIAN); else PM_PL(float, 4, PMCMC_GAUSSIAN); }
        else if (D <= 8) { if (f64) PM_PL(double, 8, PMCMC_GAUSSIAN); else PM_PL(float, 8, PMCMC_GAUSSIAN); }
        else return set_error(c, PMCMC_EUNSUPPORTED, "parallel leapfrog Gaussian supports D <= 8");
    }
#undef PM_PL
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(c, PMCMC_ECUDA, cudaGetErrorString(e));
    cudaEventRecord(c->ev1, st);
    e = cudaMemcpyAsync(c->host_ctl, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(c, PMCMC_ECUDA, cudaGetErrorString(e));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    if (res) {
        res->iters = (int)std::min<unsigned long long>(c->host_ctl->inner_iters, 0x7fffffffull);
        res->status = PMCMC_OK;
        res->max_residual = 0.0;
        res->accept_rate = (double)c->host_ctl->stats[0].accepts / (double)T;
        res->min_margin = ord_decode(c->host_ctl->stats[0].min_margin);
        res->elapsed_ms = ms;
    }
    return PMCMC_OK;
}

}  // namespace pm
