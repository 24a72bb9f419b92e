// Fused evaluate-and-linearise pass for targets whose per-step state fits in registers
// (Gaussian with D <= 32, banana).  One thread per timestep t evaluates f_t(s_{t-1}) and the
// Newton Jacobian at once, writes the scan's affine pair (J_t, r_t = f_t - s_t) and reduces the
// residual statistics.  Also the sequential chain (the paper's sequential baseline).
//
// Transitions:
//   MALA (Section 3.2):  x~ = x + eps g(x) + sqrt(2 eps) xi,  ell = log p(x~) - log p(x)
//       + log q(x | x~) - log q(x~ | x); log q(x~ | x) = -|xi|^2/2 once xi is fixed.
//   HMC (Algorithm 2, sequential leapfrog): v0 = xi, half step, L leapfrogs, negative half step.
//   Accept iff min(0, ell) - log u > 0 (min propagates NaN, so a divergent proposal rejects).
//   ell and the comparison are evaluated in FP64.
// Jacobian under the stop-gradient gate of Section 3.2:
//   J = g dprop/dx + (1 - g) I + sigma'(g~) (prop - x) (grad g~)^T,  grad g~ = 1(ell<0) grad ell.
//   MALA: dprop/dx = I + eps H(x);  grad ell = v + eps H(x) v - g - e / (2 eps) with
//         e = x - x~ - eps g(x~), v = g(x~) + (e + eps H(x~) e) / (2 eps).
//   HMC:  forward tangents through the leapfrog: J z = g dx_L + (1-g) z + sigma' (x_L - x0)
//         d(H0 - HL)[z], d(H0 - HL)[z] = -g(x0).z - v_L.dv_L + g(x_L).dx_L.
//   DIAG: exact diagonal (Eq. 4); DIAG_HUTCH: z (.) J z with Rademacher z (Eq. 9);
//   DENSE: all of J (Eq. 2); ZERO: J = 0.  Then J <- clip(damping J) (App. B.4).
#pragma once

#include "common.cuh"
#include "eval.h"
#include "targets.cuh"

namespace pm {

namespace {

template <typename R>
__device__ __forceinline__ R post_j(R v, R damping, int clip) {
    v *= damping;
    if (clip) v = v > R(1) ? R(1) : (v < R(-1) ? R(-1) : v);
    return v;
}

__device__ __forceinline__ double dsigmoid(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 - s);
}

// Rademacher probe for (t, d) at Newton iteration `iter`: Philox counter (0, t, chain, 2+iter).
__device__ __forceinline__ uint4 probe_bits(unsigned long long seed, unsigned int chain, int t,
                                            int iter) {
    return philox4x32_10(make_uint4(0u, (unsigned int)t, chain, 2u + (unsigned int)iter),
                         make_uint2((unsigned int)seed, (unsigned int)(seed >> 32)));
}
__device__ __forceinline__ float probe_sign(uint4 w, int d) {
    unsigned int word = d < 32 ? w.x : (d < 64 ? w.y : (d < 96 ? w.z : w.w));
    return ((word >> (d & 31)) & 1u) ? 1.0f : -1.0f;
}

// ------------------------------------------------------------------------------------------
// MALA
// ------------------------------------------------------------------------------------------
template <typename R, int DM, class TG>
struct MalaState {
    R x[DM], g[DM], xt[DM], gt[DM], e[DM], gl[DM];
    bool acc;
    double ell, gtl;
    R cg;  // sigma'(g~) when the gate term is active, else 0
};

template <typename R, int DM, class TG>
__device__ __forceinline__ void mala_forward(const TG &tg, R eps, const R *x, const R *xi,
                                             double u, bool want_gate,
                                             MalaState<R, DM, TG> &m) {
#pragma unroll
    for (int d = 0; d < DM; d++) m.x[d] = x[d];
    tg.grad(m.x, m.g);
    const R sq = sqrt(R(2) * eps);
#pragma unroll
    for (int d = 0; d < DM; d++) m.xt[d] = m.x[d] + eps * m.g[d] + sq * xi[d];
    tg.grad(m.xt, m.gt);
    const double lx = tg.logp(m.x, m.g), lxt = tg.logp(m.xt, m.gt);
    double ee = 0.0, xx = 0.0;
#pragma unroll
    for (int d = 0; d < DM; d++) {
        m.e[d] = m.x[d] - m.xt[d] - eps * m.gt[d];
        ee += (double)m.e[d] * (double)m.e[d];
        xx += (double)xi[d] * (double)xi[d];
    }
    m.ell = (lxt - lx) - ee / (4.0 * (double)eps) + 0.5 * xx;
    const double la = (m.ell < 0.0 || isnan(m.ell)) ? m.ell : 0.0;
    m.gtl = la - log(u);
    m.acc = m.gtl > 0.0;
    m.cg = R(0);
    if (want_gate && m.ell < 0.0) {
        m.cg = (R)dsigmoid(m.gtl);
        R tmp[DM], v[DM];
        tg.hvp(m.xt, m.e, tmp);
        const R inv2e = R(1) / (R(2) * eps);
#pragma unroll
        for (int d = 0; d < DM; d++) v[d] = m.gt[d] + (m.e[d] + eps * tmp[d]) * inv2e;
        tg.hvp(m.x, v, tmp);
#pragma unroll
        for (int d = 0; d < DM; d++) m.gl[d] = v[d] + eps * tmp[d] - m.g[d] - m.e[d] * inv2e;
    } else {
#pragma unroll
        for (int d = 0; d < DM; d++) m.gl[d] = R(0);
    }
}

// ------------------------------------------------------------------------------------------
// HMC (full transition, sequential leapfrog inside f_t)
// ------------------------------------------------------------------------------------------
template <typename R, int DM>
struct HmcState {
    R x0[DM], g0[DM], xL[DM];
    bool acc;
    double diff, gtl;
    R cg;
};

template <typename R, int DM, class TG>
__device__ __forceinline__ void hmc_forward(const TG &tg, R eps, int L, const R *x0,
                                            const R *xi, double u, bool want_gate,
                                            HmcState<R, DM> &h) {
    R v[DM], g[DM];
#pragma unroll
    for (int d = 0; d < DM; d++) {
        h.x0[d] = x0[d];
        h.xL[d] = x0[d];
        v[d] = xi[d];
    }
    tg.grad(h.x0, h.g0);
    double vv = 0.0;
#pragma unroll
    for (int d = 0; d < DM; d++) vv += (double)v[d] * (double)v[d];
    const double H0 = 0.5 * vv - tg.logp(h.x0, h.g0);
    const R he = R(0.5) * eps;
#pragma unroll
    for (int d = 0; d < DM; d++) {
        v[d] += he * h.g0[d];
        g[d] = h.g0[d];
    }
    for (int k = 0; k < L; k++) {
#pragma unroll
        for (int d = 0; d < DM; d++) h.xL[d] += eps * v[d];
        tg.grad(h.xL, g);
#pragma unroll
        for (int d = 0; d < DM; d++) v[d] += eps * g[d];
    }
    vv = 0.0;
#pragma unroll
    for (int d = 0; d < DM; d++) {
        v[d] -= he * g[d];
        vv += (double)v[d] * (double)v[d];
    }
    const double HL = 0.5 * vv - tg.logp(h.xL, g);
    h.diff = H0 - HL;
    const double la = (h.diff < 0.0 || isnan(h.diff)) ? h.diff : 0.0;
    h.gtl = la - log(u);
    h.acc = h.gtl > 0.0;
    h.cg = (want_gate && h.diff < 0.0) ? (R)dsigmoid(h.gtl) : R(0);
}

// J z for HMC by one forward tangent pass through the leapfrog.
template <typename R, int DM, class TG>
__device__ __forceinline__ void hmc_jvp(const TG &tg, R eps, int L, const R *xi,
                                        const HmcState<R, DM> &h, const R *z, R *Jz) {
    R X[DM], V[DM], dX[DM], dV[DM], G[DM], tmp[DM];
    const R he = R(0.5) * eps;
    tg.hvp(h.x0, z, tmp);
#pragma unroll
    for (int d = 0; d < DM; d++) {
        X[d] = h.x0[d];
        V[d] = xi[d] + he * h.g0[d];
        dX[d] = z[d];
        dV[d] = he * tmp[d];
        G[d] = h.g0[d];
    }
    for (int k = 0; k < L; k++) {
#pragma unroll
        for (int d = 0; d < DM; d++) {
            X[d] += eps * V[d];
            dX[d] += eps * dV[d];
        }
        tg.grad(X, G);
        tg.hvp(X, dX, tmp);
#pragma unroll
        for (int d = 0; d < DM; d++) {
            V[d] += eps * G[d];
            dV[d] += eps * tmp[d];
        }
    }
    tg.hvp(X, dX, tmp);
    R dgt = R(0);
#pragma unroll
    for (int d = 0; d < DM; d++) {
        V[d] -= he * G[d];
        dV[d] -= he * tmp[d];
        dgt += -h.g0[d] * z[d] - V[d] * dV[d] + G[d] * dX[d];
    }
#pragma unroll
    for (int d = 0; d < DM; d++)
        Jz[d] = (h.acc ? dX[d] : z[d]) + h.cg * (h.xL[d] - h.x0[d]) * dgt;
}

template <typename R, int DM, int TGT>
struct TargetSel;
template <typename R, int DM>
struct TargetSel<R, DM, PMCMC_GAUSSIAN> {
    using type = GaussianT<R, DM>;
};
template <typename R, int DM>
struct TargetSel<R, DM, PMCMC_BANANA> {
    using type = BananaT<R, DM>;
};

// Block reduction of the per-thread residual statistics into `st`.
__device__ __forceinline__ void reduce_stats(EvalStats *st, double err, double rmax,
                                             double margin, int acc) {
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    err = warp_max(err);
    rmax = warp_max(rmax);
    margin = warp_min(margin);
    double a = warp_sum((double)acc);
    if (lane == 0) {
        red[0][w] = err;
        red[1][w] = rmax;
        red[2][w] = margin;
        red[3][w] = a;
    }
    __syncthreads();
    if (w == 0) {
        err = lane < nw ? red[0][lane] : -INFINITY;
        rmax = lane < nw ? red[1][lane] : 0.0;
        margin = lane < nw ? red[2][lane] : INFINITY;
        a = lane < nw ? red[3][lane] : 0.0;
        err = warp_max(err);
        rmax = warp_max(rmax);
        margin = warp_min(margin);
        a = warp_sum(a);
        if (lane == 0) {
            atomic_max_d(&st->err, err);
            atomic_max_d(&st->rmax, rmax);
            atomic_min_d(&st->min_margin, margin);
            if (a > 0) atomicAdd(&st->accepts, (unsigned long long)(a + 0.5));
        }
    }
}

}  // namespace

// ==========================================================================================
// One evaluate-and-linearise pass: one thread per timestep.
// ==========================================================================================
template <typename R, typename S, int DM, int TGT, int SMP>
__global__ void __launch_bounds__(128) eval_small_kernel(EvalArgs A) {
    if (A.skip && *(volatile const int *)A.skip) return;
    __shared__ R smu[DM > 0 ? DM : 1];
    __shared__ R sP[DM * DM];
    const int D = A.D;
    if (TGT == PMCMC_GAUSSIAN) {
        const R *mu = (const R *)A.mu, *P = (const R *)A.P;
        for (int e = threadIdx.x; e < DM * DM; e += blockDim.x) {
            const int i = e / DM, j = e % DM;
            sP[e] = (i < D && j < D) ? P[i * D + j] : R(0);
        }
        for (int d = threadIdx.x; d < DM; d += blockDim.x) smu[d] = d < D ? mu[d] : R(0);
        __syncthreads();
    }
    using TG = typename TargetSel<R, DM, TGT>::type;
    TG tg;
    if constexpr (TGT == PMCMC_GAUSSIAN) {
        tg.mu = smu;
        tg.P = sP;
    }
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double err = -INFINITY, rmax = 0.0, margin = INFINITY;
    int acc_i = 0;
    if (t < A.T) {
        const R *s0 = (const R *)A.s0, *s = (const R *)A.s, *xin = (const R *)A.xi;
        const R eps = (R)A.eps, damping = (R)A.damping;
        const R *prev = t == 0 ? s0 : s + (size_t)(t - 1) * D;
        R x[DM], xi[DM], xc[DM], f[DM], jd[DM];
#pragma unroll
        for (int d = 0; d < DM; d++) {
            x[d] = d < D ? prev[d] : R(0);
            xi[d] = d < D ? xin[(size_t)t * D + d] : R(0);
            xc[d] = d < D ? s[(size_t)t * D + d] : R(0);
        }
        const double u = A.u[t];
        const int jac = A.jac;
        const bool want_gate = A.gate_grad && jac != PMCMC_JAC_ZERO;
        R *jdense = (jac == PMCMC_JAC_DENSE && A.a_out) ? (R *)A.a_out + (size_t)t * D * D : nullptr;
        bool acc;
        double ell;
        uint4 zbits = make_uint4(0, 0, 0, 0);
        if (jac == PMCMC_JAC_DIAG_HUTCH)
            zbits = probe_bits(A.seed, A.chain, t, A.iter ? *A.iter : 0);
        if constexpr (SMP == PMCMC_MALA) {
            MalaState<R, DM, TG> m;
            mala_forward<R, DM>(tg, eps, x, xi, u, want_gate, m);
            acc = m.acc;
            ell = m.ell;
            margin = fabs(m.gtl);
#pragma unroll
            for (int d = 0; d < DM; d++) f[d] = acc ? m.xt[d] : m.x[d];
            const R ga = acc ? R(1) : R(0);
            if (jac == PMCMC_JAC_DIAG) {
#pragma unroll
                for (int d = 0; d < DM; d++)
                    jd[d] = ga * (R(1) + eps * tg.hess(m.x, d, d)) + (R(1) - ga) +
                            m.cg * (m.xt[d] - m.x[d]) * m.gl[d];
            } else if (jac == PMCMC_JAC_DIAG_HUTCH) {
                R z[DM], Hz[DM];
                R gz = R(0);
#pragma unroll
                for (int d = 0; d < DM; d++) {
                    z[d] = d < D ? (R)probe_sign(zbits, d) : R(0);
                    gz += m.gl[d] * z[d];
                }
                tg.hvp(m.x, z, Hz);
#pragma unroll
                for (int d = 0; d < DM; d++)
                    jd[d] = z[d] * (z[d] + ga * eps * Hz[d] + m.cg * (m.xt[d] - m.x[d]) * gz);
            } else if (jac == PMCMC_JAC_DENSE) {
                if (jdense) {
                    for (int i = 0; i < D; i++)
                        for (int j = 0; j < D; j++) {
                            R v = ga * eps * tg.hess(m.x, i, j) + (i == j ? R(1) : R(0)) +
                                  m.cg * (m.xt[i] - m.x[i]) * m.gl[j];
                            jdense[i * D + j] = post_j(v, damping, A.clip);
                        }
                }
            } else {
#pragma unroll
                for (int d = 0; d < DM; d++) jd[d] = R(0);
            }
        } else {
            HmcState<R, DM> h;
            hmc_forward<R, DM>(tg, eps, A.L, x, xi, u, want_gate, h);
            acc = h.acc;
            ell = h.diff;
            margin = fabs(h.gtl);
#pragma unroll
            for (int d = 0; d < DM; d++) f[d] = acc ? h.xL[d] : h.x0[d];
            const bool trivial = !h.acc && h.cg == R(0);  // J = I exactly
            if (jac == PMCMC_JAC_DIAG || jac == PMCMC_JAC_DENSE) {
                for (int j = 0; j < D; j++) {
                    R z[DM], Jz[DM];
#pragma unroll
                    for (int d = 0; d < DM; d++) z[d] = d == j ? R(1) : R(0);
                    if (trivial) {
#pragma unroll
                        for (int d = 0; d < DM; d++) Jz[d] = z[d];
                    } else {
                        hmc_jvp<R, DM>(tg, eps, A.L, xi, h, z, Jz);
                    }
                    if (jac == PMCMC_JAC_DIAG) {
#pragma unroll
                        for (int d = 0; d < DM; d++)
                            if (d == j) jd[d] = Jz[d];
                    } else if (jdense) {
                        for (int i = 0; i < D; i++) jdense[i * D + j] = post_j(Jz[i], damping, A.clip);
                    }
                }
            } else if (jac == PMCMC_JAC_DIAG_HUTCH) {
                R z[DM], Jz[DM];
#pragma unroll
                for (int d = 0; d < DM; d++) z[d] = d < D ? (R)probe_sign(zbits, d) : R(0);
                if (trivial) {
#pragma unroll
                    for (int d = 0; d < DM; d++) Jz[d] = z[d];
                } else {
                    hmc_jvp<R, DM>(tg, eps, A.L, xi, h, z, Jz);
                }
#pragma unroll
                for (int d = 0; d < DM; d++) jd[d] = z[d] * Jz[d];
            } else {
#pragma unroll
                for (int d = 0; d < DM; d++) jd[d] = R(0);
            }
        }
        // outputs
        S *aout = (S *)A.a_out, *bout = (S *)A.b_out;
        R *fout = (R *)A.f_out;
        err = -INFINITY;
#pragma unroll
        for (int d = 0; d < DM; d++) {
            if (d < D) {
                const R r = f[d] - xc[d];
                const double ar = fabs((double)r);
                const double e = ar - A.rtol * fabs((double)xc[d]);
                err = isnan(e) ? INFINITY : max(err, e);
                rmax = isnan(ar) ? INFINITY : max(rmax, ar);
                if (bout) store_as<S, R>(bout + (size_t)t * D + d, r);
                if (aout && jac != PMCMC_JAC_DENSE)
                    store_as<S, R>(aout + (size_t)t * D + d, post_j(jd[d], damping, A.clip));
                if (fout) fout[(size_t)t * D + d] = f[d];
            }
        }
        if (A.acc_out) A.acc_out[t] = acc ? 1 : 0;
        if (A.ell_out) A.ell_out[t] = ell;
        acc_i = acc ? 1 : 0;
    }
    if (A.stats) reduce_stats(A.stats, err, rmax, margin, acc_i);
}

// ==========================================================================================
// Sequential chain on the GPU: one thread walks t = 1..T (the paper's sequential baseline).
// ==========================================================================================
template <typename R, int DM, int TGT, int SMP>
__global__ void seq_small_kernel(EvalArgs A) {
    __shared__ R smu[DM > 0 ? DM : 1];
    __shared__ R sP[DM * DM];
    const int D = A.D;
    if (TGT == PMCMC_GAUSSIAN) {
        const R *mu = (const R *)A.mu, *P = (const R *)A.P;
        for (int e = threadIdx.x; e < DM * DM; e += blockDim.x) {
            const int i = e / DM, j = e % DM;
            sP[e] = (i < D && j < D) ? P[i * D + j] : R(0);
        }
        for (int d = threadIdx.x; d < DM; d += blockDim.x) smu[d] = d < D ? mu[d] : R(0);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    using TG = typename TargetSel<R, DM, TGT>::type;
    TG tg;
    if constexpr (TGT == PMCMC_GAUSSIAN) {
        tg.mu = smu;
        tg.P = sP;
    }
    const R *xin = (const R *)A.xi;
    R *out = (R *)A.f_out;
    const R eps = (R)A.eps;
    R x[DM], xi[DM];
#pragma unroll
    for (int d = 0; d < DM; d++) x[d] = d < D ? ((const R *)A.s0)[d] : R(0);
    for (int t = 0; t < A.T; t++) {
#pragma unroll
        for (int d = 0; d < DM; d++) xi[d] = d < D ? xin[(size_t)t * D + d] : R(0);
        bool acc;
        if constexpr (SMP == PMCMC_MALA) {
            MalaState<R, DM, TG> m;
            mala_forward<R, DM>(tg, eps, x, xi, A.u[t], false, m);
            acc = m.acc;
            if (acc) {
#pragma unroll
                for (int d = 0; d < DM; d++) x[d] = m.xt[d];
            }
        } else {
            HmcState<R, DM> h;
            hmc_forward<R, DM>(tg, eps, A.L, x, xi, A.u[t], false, h);
            acc = h.acc;
            if (acc) {
#pragma unroll
                for (int d = 0; d < DM; d++) x[d] = h.xL[d];
            }
        }
        for (int d = 0; d < D; d++) out[(size_t)t * D + d] = x[d];
        if (A.acc_out) A.acc_out[t] = acc ? 1 : 0;
    }
}

// ------------------------------------------------------------------------------------------
// Dispatch
// ------------------------------------------------------------------------------------------
template <typename R, typename S, int TGT, int SMP>
cudaError_t dispatch_dm(const EvalArgs &A, cudaStream_t st, bool seq) {
    const int D = A.D;
    const int blocks = ceil_div(A.T, 128);
#define PM_CASE(DM_)                                                                   \
    if (D <= DM_) {                                                                    \
        if (seq) {                                                                     \
            seq_small_kernel<R, DM_, TGT, SMP><<<1, 32, 0, st>>>(A);                   \
        } else {                                                                       \
            prefer_shared(eval_small_kernel<R, S, DM_, TGT, SMP>);                     \
            eval_small_kernel<R, S, DM_, TGT, SMP><<<blocks, 128, 0, st>>>(A);         \
        }                                                                              \
        return cudaGetLastError();                                                     \
    }
    if constexpr (TGT == PMCMC_BANANA) {
        PM_CASE(2)
    } else {
        PM_CASE(2)
        PM_CASE(4)
        PM_CASE(8)
        PM_CASE(32)
    }
#undef PM_CASE
    return cudaErrorInvalidValue;
}

template <typename R, typename S>
cudaError_t dispatch_ts(const EvalArgs &A, cudaStream_t st, bool seq) {
    if (A.sampler == PMCMC_GIBBS) return launch_gibbs<R, S>(A, st, seq);
    if (A.target == PMCMC_GAUSSIAN) {
        if (A.sampler == PMCMC_MALA) return dispatch_dm<R, S, PMCMC_GAUSSIAN, PMCMC_MALA>(A, st, seq);
        return dispatch_dm<R, S, PMCMC_GAUSSIAN, PMCMC_HMC>(A, st, seq);
    }
    if (A.target == PMCMC_BANANA) {
        if (A.sampler == PMCMC_MALA) return dispatch_dm<R, S, PMCMC_BANANA, PMCMC_MALA>(A, st, seq);
        return dispatch_dm<R, S, PMCMC_BANANA, PMCMC_HMC>(A, st, seq);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pm
