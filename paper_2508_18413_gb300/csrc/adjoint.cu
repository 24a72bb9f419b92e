// Adjoint of a chain functional at the converged fixed point, with the accept decisions held.
//
// With every decision fixed, s_t = f_t(s_{t-1}; theta) is smooth in theta = (eps, sigma_p), and
// for L(s_1..s_T) the reverse recursion
//   lambda_T = dL/ds_T,   lambda_t = dL/ds_t + J_{t+1}^T lambda_{t+1},
//   dL/dtheta = sum_t lambda_t^T d f_t / d theta
// gives the gradient.  J_{t+1} = I + eps H(s_t) when step t+1 was accepted, else I (MALA:
// f = x~ = x + eps grad log p(x) + sqrt(2 eps) xi when accepted, f = x when rejected); H is
// symmetric, so J^T = J.  For an accepted step from x = s_{t-1}:
//   d f / d eps = grad log p(x) + xi_t / sqrt(2 eps),   d f / d sigma_p = 2 eps x / sigma_p^3.
//
// The reverse recursion is a linear recursion run backward in time, so it is solved by the
// same single-pass look-back scan as the forward Newton step, here with dense D x D maps
// (D <= 128) in reversed index order.  Rejected steps contribute identity maps, so dense J is
// built only for accepted steps (compacted).  When the accepted J's of the whole chain exceed
// the memory budget, the chain is processed in segments from the end: each segment rebuilds
// its J's, scans with the carry lambda from the later segment, and accumulates its part of
// dL/dtheta (the recompute path).
#include <vector>

#include "common.cuh"
#include "hess_tc.h"
#include "solve.h"

namespace pm {

namespace {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ unsigned int take_ticket(ScanCtl *ctl, unsigned int *s_tile,
                                                    unsigned int *s_epoch) {
    if (threadIdx.x == 0) {
        *s_tile = atomicAdd(&ctl->ticket, 1u);
        *s_epoch = *(volatile unsigned int *)&ctl->epoch;
    }
    __syncthreads();
    return *s_tile;
}

__device__ __forceinline__ void finish_ticket(ScanCtl *ctl, unsigned int ntiles) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int d = atomicAdd(&ctl->done, 1u);
        if (d == ntiles - 1) {
            ctl->ticket = 0;
            ctl->done = 0;
            ctl->epoch = ctl->epoch + 1u;
            __threadfence();
        }
    }
}

__device__ __forceinline__ unsigned int flag_of(unsigned int epoch, unsigned int st) {
    return ((epoch & 0x3fffffffu) << 2) | st;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// J_t = I + eps H(s_{t-1}) for a list of (accepted) timesteps, logistic target:
//   H = -X^T diag(w) X - I / sigma_p^2,  w_n = sigmoid(z_n)(1 - sigmoid(z_n)),  z = X s_{t-1}.
// CTA = (group of TB listed timesteps) x (64 x 64 output tile); thread = 4 x 4 outputs x TB.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) adj_hess_logreg_kernel(
    int nlist, const int *__restrict__ list, int D, int N, const R *__restrict__ X,
    const R *__restrict__ s0, const R *__restrict__ s, R eps, R inv_sp2, R *__restrict__ Jbuf) {
    constexpr int TB = 4, NC = sizeof(R) == 8 ? 16 : 32, TILE = 64;
    __shared__ R xs[TB][128];
    __shared__ R Xc[NC][TILE + 1];  // rows n, columns i of the tile (row block)
    __shared__ R Xd[NC][TILE + 1];  // rows n, columns j of the tile (column block)
    __shared__ R Xf[NC][129];       // full rows for z
    __shared__ R w[TB][NC];
    const int g0 = blockIdx.x * TB;
    const int ti = blockIdx.y, tj = blockIdx.z;
    const int i0 = ti * TILE, j0 = tj * TILE;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    for (int e = tid; e < TB * D; e += 256) {
        const int b = e / D, d = e % D;
        R v = R(0);
        if (g0 + b < nlist) {
            const int t = list[g0 + b];
            v = t == 0 ? s0[d] : s[(size_t)(t - 1) * D + d];
        }
        xs[b][d] = v;
    }
    R acc[TB][4][4];
#pragma unroll
    for (int b = 0; b < TB; b++)
#pragma unroll
        for (int p = 0; p < 4; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[b][p][q] = R(0);
    for (int n0 = 0; n0 < N; n0 += NC) {
        __syncthreads();
        for (int e = tid; e < NC * D; e += 256) {
            const int r = e / D, d = e % D;
            Xf[r][d] = (n0 + r < N) ? X[(size_t)(n0 + r) * D + d] : R(0);
        }
        __syncthreads();
        for (int e = tid; e < NC * TILE; e += 256) {
            const int r = e / TILE, c = e % TILE;
            Xc[r][c] = (i0 + c < D) ? Xf[r][i0 + c] : R(0);
            Xd[r][c] = (j0 + c < D) ? Xf[r][j0 + c] : R(0);
        }
        // w for the TB timesteps of this chunk (one thread per (b, r))
        if (tid < TB * NC) {
            const int b = tid / NC, r = tid % NC;
            R z = R(0);
            for (int d = 0; d < D; d++) z = fma(Xf[r][d], xs[b][d], z);
            const R p = R(1) / (R(1) + exp(-z));
            w[b][r] = (n0 + r < N) ? p * (R(1) - p) : R(0);
        }
        __syncthreads();
        for (int r = 0; r < NC; r++) {
            R xi[4], xj[4];
#pragma unroll
            for (int p = 0; p < 4; p++) {
                xi[p] = Xc[r][ty * 4 + p];
                xj[p] = Xd[r][tx * 4 + p];
            }
#pragma unroll
            for (int b = 0; b < TB; b++) {
                const R wb = w[b][r];
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    const R wx = wb * xi[p];
#pragma unroll
                    for (int q = 0; q < 4; q++) acc[b][p][q] = fma(wx, xj[q], acc[b][p][q]);
                }
            }
        }
    }
    const int DD = D * D;
#pragma unroll
    for (int b = 0; b < TB; b++) {
        if (g0 + b >= nlist) continue;
        R *J = Jbuf + (size_t)(g0 + b) * DD;
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const int i = i0 + ty * 4 + p;
            if (i >= D) continue;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int j = j0 + tx * 4 + q;
                if (j >= D) continue;
                const R H = -acc[b][p][q] - (i == j ? inv_sp2 : R(0));
                J[i * D + j] = eps * H + (i == j ? R(1) : R(0));
            }
        }
    }
}

// Gaussian target: J = I - eps P for every accepted step (one matrix).
template <typename R>
__global__ void adj_hess_gauss_kernel(int D, const R *__restrict__ P, R eps, R *__restrict__ J) {
    for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < D * D; e += blockDim.x * gridDim.x) {
        const int i = e / D, j = e % D;
        J[e] = (i == j ? R(1) : R(0)) - eps * P[e];
    }
}

// ------------------------------------------------------------------------------------------
// Reverse dense scan over a segment [t_lo, t_hi) with identity-aware maps.
// Local index tau = 0..n-1 stands for t = t_hi - 1 - tau; element tau is the map
//   mu -> A_tau mu + b_tau,  A_tau = J_{t+1} (identity when step t+1 was rejected or t+1 = T),
//   b_tau = dL/ds_t,  starting from mu_{-1} = carry (lambda_{t_hi}, zero for the last segment).
// Output lambda_t = mu_tau.  jmap[k - t_lo - 1] gives the J buffer slot of step k in
// (t_lo, t_hi] or -1 (identity); `shared_j` makes every accepted step use slot 0.
// ------------------------------------------------------------------------------------------
template <typename R, int DM>
__global__ void __launch_bounds__(kAdjThreads) rev_scan_dense_kernel(
    int t_lo, int t_hi, int T, int D, int C, const int *__restrict__ jmap, int shared_j,
    const R *__restrict__ Jbuf, const R *__restrict__ dLds, const R *__restrict__ carry,
    R *__restrict__ lam, unsigned int *flags, R *gagg, R *gincl, ScanCtl *ctl,
    unsigned int spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *Phi0 = reinterpret_cast<R *>(smem_raw);
    R *Phi1 = Phi0 + DM * DM;
    R *At = Phi1 + DM * DM;        // transposed A of the current step
    R *beta = At + DM * DM;        // 2 x DM
    R *vec = beta + 2 * DM;        // 2 x DM
    __shared__ unsigned int s_tile, s_epoch;
    __shared__ int s_jj, s_to;
    const int n = t_hi - t_lo;
    const unsigned int ntiles = (unsigned int)ceil_div(n, C);
    const int tile = (int)take_ticket(ctl, &s_tile, &s_epoch);
    const unsigned int epoch = s_epoch;
    const int tid = threadIdx.x;
    const int DD = D * D;
    const int c0 = tile * C, cv = min(C, n - c0);
    const size_t AGG = (size_t)DD + D;
    constexpr int MT = DM / 16;  // micro-tile of the D x D product
    const int ty = tid >> 4, tx = tid & 15;

    auto jptr = [&](int tau) -> const R * {  // A_tau, or nullptr for identity
        const int k = t_hi - tau;             // step k = t + 1
        if (k >= T) return nullptr;
        const int slot = jmap[k - t_lo - 1];
        if (slot < 0) return nullptr;
        return Jbuf + (size_t)(shared_j ? 0 : slot) * DD;
    };

    // Phase A: chunk aggregate (Phi, beta) = composition of the maps tau in [c0, c0 + cv)
    for (int e = tid; e < DM * DM; e += kAdjThreads) {
        const int i = e / DM, j = e % DM;
        Phi0[e] = (i == j && i < D) ? R(1) : R(0);
    }
    for (int d = tid; d < DM; d += kAdjThreads) beta[d] = R(0);
    __syncthreads();
    R *Pc = Phi0, *Pn = Phi1;
    for (int i = 0; i < cv; i++) {
        const int tau = c0 + i;
        const int t = t_hi - 1 - tau;
        const R *A = jptr(tau);
        if (A) {
            for (int e = tid; e < DM * DM; e += kAdjThreads) {
                const int r = e / DM, k = e % DM;
                At[k * DM + r] = (r < D && k < D) ? A[r * D + k] : R(0);
            }
            __syncthreads();
            // Pn = A Pc (micro-tile MT x MT per thread)
            R acc[MT][MT];
#pragma unroll
            for (int p = 0; p < MT; p++)
#pragma unroll
                for (int q = 0; q < MT; q++) acc[p][q] = R(0);
            for (int k = 0; k < D; k++) {
                R a[MT], bb[MT];
#pragma unroll
                for (int p = 0; p < MT; p++) a[p] = At[k * DM + ty * MT + p];
#pragma unroll
                for (int q = 0; q < MT; q++) bb[q] = Pc[k * DM + tx * MT + q];
#pragma unroll
                for (int p = 0; p < MT; p++)
#pragma unroll
                    for (int q = 0; q < MT; q++) acc[p][q] = fma(a[p], bb[q], acc[p][q]);
            }
            // beta' = A beta + b (rows)
            R nb = R(0);
            if (tid < D) {
                nb = dLds[(size_t)t * D + tid];
                for (int k = 0; k < D; k++) nb = fma(At[k * DM + tid], beta[k], nb);
            }
            __syncthreads();
#pragma unroll
            for (int p = 0; p < MT; p++)
#pragma unroll
                for (int q = 0; q < MT; q++) Pn[(ty * MT + p) * DM + tx * MT + q] = acc[p][q];
            if (tid < D) beta[tid] = nb;
            __syncthreads();
            R *tmp = Pc;
            Pc = Pn;
            Pn = tmp;
        } else {
            if (tid < D) beta[tid] += dLds[(size_t)t * D + tid];
            __syncthreads();
        }
    }
    // Phase C: publish, look back, publish inclusive
    if (tile == 0) {
        // inclusive of tile 0 = Phi carry + beta
        if (tid < D) {
            R acc = beta[tid];
            if (carry)
                for (int k = 0; k < D; k++) acc = fma(Pc[tid * DM + k], carry[k], acc);
            gincl[tid] = acc;
            vec[tid] = carry ? carry[tid] : R(0);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(flags, flag_of(epoch, 2));
    } else {
        for (int e = tid; e < DD; e += kAdjThreads) {
            const int i = e / D, j = e % D;
            gagg[(size_t)tile * AGG + e] = Pc[i * DM + j];
        }
        if (tid < D) gagg[(size_t)tile * AGG + DD + tid] = beta[tid];
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            st_release(flags + tile, flag_of(epoch, 1));
            int jj = tile - 1;
            int to = 0;
            for (; jj >= 0; jj--) {
                Spin spin(spin_limit);
                unsigned int st = 0;
                for (;;) {
                    unsigned int f = ld_acquire(flags + jj);
                    if ((f >> 2) == (epoch & 0x3fffffffu) && (f & 3u)) {
                        st = f & 3u;
                        break;
                    }
                    if (!spin.again()) {
                        atomicExch(&ctl->timeout, 1u);
                        break;
                    }
                }
                if (st == 2 || st == 0) {
                    to = st == 0;
                    break;
                }
            }
            s_jj = jj;
            s_to = to;
        }
        __syncthreads();
        const int jj = s_jj;
        const bool timed_out = s_to != 0;  // carry from zero; the status reports the timeout
        int vc = 0;
        if (tid < D) vec[tid] = (!timed_out && jj >= 0) ? gincl[(size_t)jj * D + tid] : R(0);
        __syncthreads();
        for (int m = jj + 1; m < tile; m++) {
            const R *Am = gagg + (size_t)m * AGG;
            R acc = R(0);
            if (tid < D) {
                acc = Am[DD + tid];
                for (int k = 0; k < D; k++) acc = fma(Am[tid * D + k], vec[vc * DM + k], acc);
                vec[(vc ^ 1) * DM + tid] = acc;
            }
            __syncthreads();
            vc ^= 1;
        }
        if (tid < D) {
            R acc = beta[tid];
            for (int k = 0; k < D; k++) acc = fma(Pc[tid * DM + k], vec[vc * DM + k], acc);
            gincl[(size_t)tile * D + tid] = acc;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(flags + tile, flag_of(epoch, 2));
        if (vc == 1 && tid < D) vec[tid] = vec[DM + tid];
        __syncthreads();
    }
    // Phase D: mu_tau = A_tau mu_{tau-1} + b_tau from the carry; write lambda
    int vc = 0;
    for (int i = 0; i < cv; i++) {
        const int tau = c0 + i;
        const int t = t_hi - 1 - tau;
        const R *A = jptr(tau);
        if (tid < D) {
            R acc = dLds[(size_t)t * D + tid];
            if (A) {
                for (int k = 0; k < D; k++) acc = fma(A[tid * D + k], vec[vc * DM + k], acc);
            } else {
                acc += vec[vc * DM + tid];
            }
            vec[(vc ^ 1) * DM + tid] = acc;
            lam[(size_t)t * D + tid] = acc;
        }
        __syncthreads();
        vc ^= 1;
    }
    finish_ticket(ctl, ntiles);
}

// ------------------------------------------------------------------------------------------
// dL/dtheta contributions of accepted steps: lambda_t . (grad log p(x) + xi_t / sqrt(2 eps))
// and lambda_t . (2 eps x / sigma_p^3), x = s_{t-1}.  One CTA per TB listed steps.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) adj_theta_kernel(
    int nlist, const int *__restrict__ list, int target, int D, int N, const R *__restrict__ X,
    const R *__restrict__ y, const R *__restrict__ mu, const R *__restrict__ P,
    const R *__restrict__ s0, const R *__restrict__ s, const R *__restrict__ xi,
    const R *__restrict__ lam, double eps, double sigma_p, double *out) {
    constexpr int TB = 8, NC = sizeof(R) == 8 ? 16 : 64;
    __shared__ R xs[TB][128];
    __shared__ R g[TB][128];
    __shared__ R Xc[NC][129];
    __shared__ R cc[TB][NC];
    const int g0 = blockIdx.x * TB;
    const int tid = threadIdx.x;
    for (int e = tid; e < TB * 128; e += 256) {
        const int b = e / 128, d = e % 128;
        R v = R(0);
        if (g0 + b < nlist && d < D) {
            const int t = list[g0 + b];
            v = t == 0 ? s0[d] : s[(size_t)(t - 1) * D + d];
        }
        xs[b][d] = v;
        g[b][d] = R(0);
    }
    __syncthreads();
    if (target == PMCMC_LOGREG) {
        for (int n0 = 0; n0 < N; n0 += NC) {
            __syncthreads();
            for (int e = tid; e < NC * D; e += 256) {
                const int r = e / D, d = e % D;
                Xc[r][d] = (n0 + r < N) ? X[(size_t)(n0 + r) * D + d] : R(0);
            }
            __syncthreads();
            for (int e = tid; e < TB * NC; e += 256) {
                const int b = e / NC, r = e % NC;
                R z = R(0);
                for (int d = 0; d < D; d++) z = fma(Xc[r][d], xs[b][d], z);
                const R p = R(1) / (R(1) + exp(-z));
                cc[b][r] = (n0 + r < N) ? y[n0 + r] - p : R(0);
            }
            __syncthreads();
            for (int e = tid; e < TB * D; e += 256) {
                const int b = e / D, d = e % D;
                R acc = g[b][d];
                for (int r = 0; r < NC; r++) acc = fma(cc[b][r], Xc[r][d], acc);
                g[b][d] = acc;
            }
        }
        __syncthreads();
        for (int e = tid; e < TB * D; e += 256) {
            const int b = e / D, d = e % D;
            g[b][d] -= xs[b][d] / (R)(sigma_p * sigma_p);
        }
    } else {
        for (int e = tid; e < TB * D; e += 256) {
            const int b = e / D, d = e % D;
            R acc = R(0);
            for (int k = 0; k < D; k++) acc = fma(P[d * D + k], xs[b][k] - mu[k], acc);
            g[b][d] = -acc;
        }
    }
    __syncthreads();
    double c_eps = 0.0, c_sp = 0.0;
    const double inv = 1.0 / sqrt(2.0 * eps);
    for (int e = tid; e < TB * D; e += 256) {
        const int b = e / D, d = e % D;
        if (g0 + b >= nlist) continue;
        const int t = list[g0 + b];
        const double l = (double)lam[(size_t)t * D + d];
        c_eps += l * ((double)g[b][d] + (double)xi[(size_t)t * D + d] * inv);
        if (target == PMCMC_LOGREG) c_sp += l * 2.0 * eps * (double)xs[b][d] / (sigma_p * sigma_p * sigma_p);
    }
    c_eps = warp_sum(c_eps);
    c_sp = warp_sum(c_sp);
    if ((tid & 31) == 0) {
        atomicAdd(&out[0], c_eps);
        atomicAdd(&out[1], c_sp);
    }
}

}  // namespace pm

using namespace pm;

template <typename R, int DM>
static cudaError_t launch_rev_scan(int t_lo, int t_hi, int T, int D, int C, const int *jmap,
                                   int shared_j, const void *Jbuf, const void *dLds,
                                   const void *carry, void *lam, const ScanWork &w,
                                   unsigned int spin, cudaStream_t st) {
    const size_t sm = sizeof(R) * ((size_t)3 * DM * DM + 4 * DM);
    auto k = rev_scan_dense_kernel<R, DM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<ceil_div(t_hi - t_lo, C), kAdjThreads, sm, st>>>(
        t_lo, t_hi, T, D, C, jmap, shared_j, (const R *)Jbuf, (const R *)dLds, (const R *)carry,
        (R *)lam, w.flags, (R *)w.agg, (R *)w.incl, w.ctl, spin);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t rev_scan(int t_lo, int t_hi, int T, int D, int C, const int *jmap,
                            int shared_j, const void *Jbuf, const void *dLds, const void *carry,
                            void *lam, const ScanWork &w, unsigned int spin, cudaStream_t st) {
    if (D <= 32)
        return launch_rev_scan<R, 32>(t_lo, t_hi, T, D, C, jmap, shared_j, Jbuf, dLds, carry, lam, w, spin, st);
    if (D <= 64)
        return launch_rev_scan<R, 64>(t_lo, t_hi, T, D, C, jmap, shared_j, Jbuf, dLds, carry, lam, w, spin, st);
    if (sizeof(R) == 8) return cudaErrorInvalidValue;
    return launch_rev_scan<R, 128>(t_lo, t_hi, T, D, C, jmap, shared_j, Jbuf, dLds, carry, lam, w, spin, st);
}

#define PM_CUDA_A(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return set_error(c, PMCMC_ECUDA, cudaGetErrorString(e_));      \
    } while (0)

extern "C" pmcmc_status pmcmc_adjoint(pmcmc_ctx *c, const pmcmc_target *tg,
                                      const pmcmc_options *o, int T, const void *s0,
                                      const void *s, const unsigned char *acc, const void *xi,
                                      const double *u, const void *dL_ds,
                                      size_t jac_budget_bytes, void *lambda_out,
                                      double *grad_out, void *stream) {
    (void)u;
    if (!c) return PMCMC_EINVAL;
    if (!tg || !o || !s0 || !s || !acc || !xi || !dL_ds || !grad_out)
        return set_error(c, PMCMC_EINVAL, "adjoint: null argument");
    if (o->sampler != PMCMC_MALA) return set_error(c, PMCMC_EUNSUPPORTED, "adjoint: MALA only");
    if (tg->kind != PMCMC_LOGREG && tg->kind != PMCMC_GAUSSIAN)
        return set_error(c, PMCMC_EUNSUPPORTED, "adjoint: logistic or Gaussian targets");
    const int D = tg->D;
    const bool f64 = o->precision == PMCMC_F64;
    if (D <= 0 || D > 128 || (f64 && D > 64))
        return set_error(c, PMCMC_EUNSUPPORTED, "adjoint: D <= 128 (FP32) or 64 (FP64)");
    if (o->precision == PMCMC_F32_SCAN_BF16) return set_error(c, PMCMC_EINVAL, "adjoint: F32 or F64");
    if (tg->kind == PMCMC_LOGREG && (!tg->X || !tg->y || tg->N <= 0))
        return set_error(c, PMCMC_EINVAL, "adjoint: logistic target needs X and y");
    if (tg->kind == PMCMC_GAUSSIAN && (!tg->mean || !tg->prec))
        return set_error(c, PMCMC_EINVAL, "adjoint: Gaussian target needs mean and prec");
    grad_out[0] = grad_out[1] = 0.0;
    if (T == 0) return PMCMC_OK;
    PM_CUDA_A(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int rb = f64 ? 8 : 4;
    const size_t DD = (size_t)D * D;

    // decisions to the host: the accepted steps and their compacted order
    std::vector<unsigned char> hacc(T);
    PM_CUDA_A(cudaMemcpyAsync(hacc.data(), acc, T, cudaMemcpyDeviceToHost, st));
    PM_CUDA_A(cudaStreamSynchronize(st));
    std::vector<int> accepted;
    accepted.reserve(T);
    for (int t = 0; t < T; t++)
        if (hacc[t]) accepted.push_back(t);
    const bool gauss = tg->kind == PMCMC_GAUSSIAN;
    // segments from the end, each holding at most `cap` accepted J's
    size_t cap = accepted.size();
    if (!gauss && jac_budget_bytes > 0) cap = std::max<size_t>(1, jac_budget_bytes / (DD * rb));
    if (gauss) cap = std::max<size_t>(cap, 1);
    std::vector<std::pair<int, int>> segs;  // [t_lo, t_hi)
    {
        int t_hi = T;
        // J of step k is needed for k in (t_lo, t_hi]; count accepted k in that range
        while (t_hi > 0) {
            int t_lo = t_hi - 1;
            size_t cnt = (t_hi < T && hacc[t_hi]) ? 1 : 0;
            while (t_lo > 0) {
                const size_t add = hacc[t_lo] ? 1 : 0;
                if (!gauss && cnt + add > cap) break;
                cnt += add;
                t_lo--;
            }
            segs.push_back({t_lo, t_hi});
            t_hi = t_lo;
        }
    }
    // workspace: lambda (T x D), J slots, jmap, list, scan work, carry, theta accumulators
    int max_seg = 1;
    for (auto &sg : segs) max_seg = std::max(max_seg, sg.second - sg.first);
    const int C = std::max(8, std::min(64, ceil_div(max_seg, 2 * 152)));
    const int max_tiles = ceil_div(max_seg, C);
    const size_t jslots = gauss ? 1 : std::min(cap, accepted.size() + 1);
    Carve cv;
    const size_t o_lam = cv.take((size_t)rb * T * D);
    const size_t o_j = cv.take((size_t)rb * DD * std::max<size_t>(jslots, 1));
    const size_t o_jmap = cv.take(sizeof(int) * (size_t)max_seg);
    const size_t o_list = cv.take(sizeof(int) * std::max<size_t>(accepted.size(), 1));
    const size_t o_flags = cv.take(sizeof(unsigned int) * max_tiles);
    const size_t o_agg = cv.take((size_t)rb * max_tiles * (DD + D));
    const size_t o_incl = cv.take((size_t)rb * max_tiles * D);
    const size_t o_theta = cv.take(2 * sizeof(double));
    // 64 < D <= 128, FP32: the J's are formed on the tensor cores from an image of X^T
    const bool hess_tc = !gauss && !f64 && o->engine != 1 && hess_tc_supported(D, tg->N);
    const size_t o_img = hess_tc ? cv.take(hess_tc_image_bytes(tg->N)) : 0;
    const size_t o_w = hess_tc ? cv.take(sizeof(float) * hess_tc_w_floats((int)jslots, tg->N)) : 0;
    pmcmc_status ps = ws_reserve(c, cv.used);
    if (ps != PMCMC_OK) return ps;
    char *base = (char *)c->ws;
    void *lam = lambda_out ? lambda_out : (void *)(base + o_lam), *Jbuf = base + o_j;
    int *jmap_d = (int *)(base + o_jmap), *list_d = (int *)(base + o_list);
    double *theta = (double *)(base + o_theta);
    ScanWork w;
    w.flags = (unsigned int *)(base + o_flags);
    w.agg = base + o_agg;
    w.incl = base + o_incl;
    w.max_tiles = max_tiles;
    w.ctl = &c->ctl->scan;
    PM_CUDA_A(cudaMemsetAsync(w.flags, 0, sizeof(unsigned int) * max_tiles, st));
    c->flags_generation = ~0ull;  // the solver re-zeroes its own flag area next time
    PM_CUDA_A(cudaMemsetAsync(theta, 0, 2 * sizeof(double), st));
    if (!accepted.empty())
        PM_CUDA_A(cudaMemcpyAsync(list_d, accepted.data(), sizeof(int) * accepted.size(),
                                  cudaMemcpyHostToDevice, st));
    const unsigned int spin = o->spin_limit > 0 ? (unsigned int)o->spin_limit : kDefaultSpinLimit;
    const double eps = o->step, sp = tg->prior_scale > 0 ? tg->prior_scale : 1.0;
    if (gauss) {
        if (f64)
            adj_hess_gauss_kernel<double><<<ceil_div(DD, 256), 256, 0, st>>>(D, (const double *)tg->prec, eps, (double *)Jbuf);
        else
            adj_hess_gauss_kernel<float><<<ceil_div(DD, 256), 256, 0, st>>>(D, (const float *)tg->prec, (float)eps, (float *)Jbuf);
        PM_CUDA_A(cudaGetLastError());
    }
    if (hess_tc)
        PM_CUDA_A(launch_hess_tc_pack((const float *)tg->X, tg->N, D, base + o_img, st));
    std::vector<int> jmap(max_seg);
    // the accepted list is sorted; locate each segment's range by binary search
    for (size_t si = 0; si < segs.size(); si++) {
        const int t_lo = segs[si].first, t_hi = segs[si].second;
        const int n = t_hi - t_lo;
        // steps k in (t_lo, t_hi] with a J: accepted k < T
        auto lo_it = std::upper_bound(accepted.begin(), accepted.end(), t_lo);
        auto hi_it = std::upper_bound(accepted.begin(), accepted.end(), std::min(t_hi, T - 1));
        const int first = (int)(lo_it - accepted.begin());
        const int cnt = (int)(hi_it - lo_it);
        for (int i = 0; i < n; i++) jmap[i] = -1;
        for (int i = 0; i < cnt; i++) jmap[accepted[first + i] - t_lo - 1] = i;
        PM_CUDA_A(cudaMemcpyAsync(jmap_d, jmap.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        if (hess_tc && cnt > 0) {
            PM_CUDA_A(launch_hess_logreg_tc(cnt, list_d + first, D, tg->N, (const float *)tg->X,
                                            base + o_img, (const float *)s0, (const float *)s,
                                            (float *)(base + o_w), (float)eps,
                                            (float)(1.0 / (sp * sp)), (float *)Jbuf,
                                            &c->ctl->scan.timeout, spin, st));
        } else if (!gauss && cnt > 0) {
            dim3 grid(ceil_div(cnt, 4), ceil_div(D, 64), ceil_div(D, 64));
            if (f64)
                adj_hess_logreg_kernel<double><<<grid, 256, 0, st>>>(
                    cnt, list_d + first, D, tg->N, (const double *)tg->X, (const double *)s0,
                    (const double *)s, eps, 1.0 / (sp * sp), (double *)Jbuf);
            else
                adj_hess_logreg_kernel<float><<<grid, 256, 0, st>>>(
                    cnt, list_d + first, D, tg->N, (const float *)tg->X, (const float *)s0,
                    (const float *)s, (float)eps, (float)(1.0 / (sp * sp)), (float *)Jbuf);
            PM_CUDA_A(cudaGetLastError());
        }
        const void *carry = t_hi < T ? (const void *)((char *)lam + (size_t)rb * t_hi * D) : nullptr;
        cudaError_t e = f64 ? rev_scan<double>(t_lo, t_hi, T, D, C, jmap_d, gauss ? 1 : 0, Jbuf,
                                               dL_ds, carry, lam, w, spin, st)
                            : rev_scan<float>(t_lo, t_hi, T, D, C, jmap_d, gauss ? 1 : 0, Jbuf,
                                              dL_ds, carry, lam, w, spin, st);
        PM_CUDA_A(e);
        // theta contributions of the accepted steps t in [t_lo, t_hi)
        auto a_it = std::lower_bound(accepted.begin(), accepted.end(), t_lo);
        auto b_it = std::lower_bound(accepted.begin(), accepted.end(), t_hi);
        const int f2 = (int)(a_it - accepted.begin()), n2 = (int)(b_it - a_it);
        if (n2 > 0) {
            if (f64)
                adj_theta_kernel<double><<<ceil_div(n2, 8), 256, 0, st>>>(
                    n2, list_d + f2, tg->kind, D, tg->N, (const double *)tg->X, (const double *)tg->y,
                    (const double *)tg->mean, (const double *)tg->prec, (const double *)s0,
                    (const double *)s, (const double *)xi, (const double *)lam, eps, sp, theta);
            else
                adj_theta_kernel<float><<<ceil_div(n2, 8), 256, 0, st>>>(
                    n2, list_d + f2, tg->kind, D, tg->N, (const float *)tg->X, (const float *)tg->y,
                    (const float *)tg->mean, (const float *)tg->prec, (const float *)s0,
                    (const float *)s, (const float *)xi, (const float *)lam, eps, sp, theta);
            PM_CUDA_A(cudaGetLastError());
        }
        // jmap is reused by the next segment: wait for this segment's kernels
        PM_CUDA_A(cudaStreamSynchronize(st));
    }
    double h[2];
    PM_CUDA_A(cudaMemcpyAsync(h, theta, sizeof(h), cudaMemcpyDeviceToHost, st));
    CtlBlock *hc = c->host_ctl;
    PM_CUDA_A(cudaMemcpyAsync(hc, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st));
    PM_CUDA_A(cudaStreamSynchronize(st));
    if (hc->scan.timeout) {
        unsigned int zero = 0;
        cudaMemcpy(&c->ctl->scan.timeout, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        return set_error(c, PMCMC_ETIMEOUT, "adjoint: a bounded wait (look-back or Jacobian pipeline) ran out");
    }
    grad_out[0] = h[0];
    grad_out[1] = h[1];
    return PMCMC_OK;
}
