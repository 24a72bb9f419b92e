// Orthogonal reparameterisation for quasi-DEER (Section 3.4, Eq. 10): the Newton solve runs on
// z_t = Q^T s_t with f^_t(z) = Q^T f_t(Q z), whose Jacobian is Q^T J_t Q, and the result is
// mapped back with s_t = Q z_t.  For MALA and HMC the rotated chain is the same chain: the
// target becomes p(Q z) (Gaussian: mean Q^T mu, precision Q^T P Q; logistic: design X Q, the
// isotropic prior unchanged) and the isotropic noise is rotated with it, xi^_t = Q^T xi_t, so
// every proposal, MH ratio and decision is unchanged.  Only the Newton iterations differ: with
// Q the eigenvectors of P a Gaussian's Q^T J Q is diagonal, and the diagonal Jacobian is exact.
#include <vector>

#include "common.cuh"
#include "solve.h"

namespace pm {

// dst[r][d] = sum_k Qop[d][k] src[r][k],  Qop = Q^T (transpose) or Q.  Q staged in shared memory.
template <typename R>
__global__ void __launch_bounds__(256) rot_rows_kernel(R *__restrict__ dst, const R *__restrict__ src,
                                                       const R *__restrict__ Q, long long rows, int D,
                                                       int transpose) {
    extern __shared__ __align__(16) unsigned char smem[];
    R *q = reinterpret_cast<R *>(smem);  // q[d * D + k] = Qop[d][k]
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
        const int d = e / D, k = e % D;
        q[e] = transpose ? Q[k * D + d] : Q[d * D + k];
    }
    __syncthreads();
    const long long n = rows * D;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / D;
        const int d = (int)(i - r * D);
        const R *x = src + r * D;
        R acc = R(0);
        for (int k = 0; k < D; k++) acc = fma(q[d * D + k], x[k], acc);
        dst[i] = acc;
    }
}

// P^ = Q^T P Q (D x D), one thread per entry
template <typename R>
__global__ void rot_sym_kernel(R *__restrict__ out, const R *__restrict__ P, const R *__restrict__ Q,
                               int D) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D * D) return;
    const int i = e / D, j = e % D;
    R acc = R(0);
    for (int a = 0; a < D; a++) {
        R pq = R(0);
        for (int b = 0; b < D; b++) pq = fma(P[a * D + b], Q[b * D + j], pq);
        acc = fma(Q[a * D + i], pq, acc);
    }
    out[e] = acc;
}

cudaError_t rot_rows(void *dst, const void *src, const void *Q, long long rows, int D,
                     bool transpose, bool f64, cudaStream_t st) {
    const size_t sm = (size_t)D * D * (f64 ? 8 : 4);
    long long n = rows * D;
    int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    if (grid < 1) grid = 1;
    if (f64) {
        auto k = rot_rows_kernel<double>;
        ensure_dyn_smem(k, sm);
        k<<<grid, 256, sm, st>>>((double *)dst, (const double *)src, (const double *)Q, rows, D, transpose);
    } else {
        auto k = rot_rows_kernel<float>;
        ensure_dyn_smem(k, sm);
        k<<<grid, 256, sm, st>>>((float *)dst, (const float *)src, (const float *)Q, rows, D, transpose);
    }
    return cudaGetLastError();
}

cudaError_t rot_sym(void *out, const void *P, const void *Q, int D, bool f64, cudaStream_t st) {
    const int blocks = ceil_div(D * D, 256);
    if (f64)
        rot_sym_kernel<double><<<blocks, 256, 0, st>>>((double *)out, (const double *)P, (const double *)Q, D);
    else
        rot_sym_kernel<float><<<blocks, 256, 0, st>>>((float *)out, (const float *)P, (const float *)Q, D);
    return cudaGetLastError();
}

pmcmc_status aux_reserve(pmcmc_ctx *c, size_t bytes) {
    if (bytes <= c->aux_bytes) return PMCMC_OK;
    if (c->aux) cudaFree(c->aux);
    c->aux = nullptr;
    c->aux_bytes = 0;
    if (cudaMalloc(&c->aux, bytes + bytes / 4) != cudaSuccess) {
        cudaGetLastError();
        return set_error(c, PMCMC_ENOMEM, "reparameterisation buffer allocation failed");
    }
    c->aux_bytes = bytes + bytes / 4;
    return PMCMC_OK;
}

#define PM_CUDA_R(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return set_error(c, PMCMC_ECUDA, cudaGetErrorString(e_));      \
    } while (0)

// pmcmc_solve with tg->Q set: rotate, solve in z, rotate back.
pmcmc_status solve_with_basis(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                              const void *s0, const void *s_init, const void *xi, const double *u,
                              void *s_out, pmcmc_result *res, void *stream) {
    if (tg->kind != PMCMC_GAUSSIAN && tg->kind != PMCMC_LOGREG)
        return set_error(c, PMCMC_EUNSUPPORTED, "the basis Q applies to Gaussian and logistic targets");
    if (o->sampler == PMCMC_HMC_PAR_LEAPFROG)
        return set_error(c, PMCMC_EUNSUPPORTED, "the basis Q is for MALA and HMC solves");
    cudaStream_t st = (cudaStream_t)stream;
    const int D = tg->D;
    const bool f64 = o->precision == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    Carve cv;
    const size_t o_xi = cv.take((size_t)rb * T * D);
    const size_t o_u = xi ? 0 : cv.take(sizeof(double) * (size_t)T);
    const size_t o_s0 = cv.take((size_t)rb * D);
    const size_t o_init = s_init ? cv.take((size_t)rb * T * D) : 0;
    const size_t o_z = cv.take((size_t)rb * T * D);
    const size_t o_mu = cv.take((size_t)rb * D);
    const size_t o_P = cv.take((size_t)rb * D * D);
    const size_t o_X = tg->kind == PMCMC_LOGREG ? cv.take((size_t)rb * tg->N * D) : 0;
    pmcmc_status ps = aux_reserve(c, cv.used);
    if (ps != PMCMC_OK) return ps;
    char *b = (char *)c->aux;
    if (!xi) {  // noise from the seed, in the original coordinates, then rotated
        PM_CUDA_R(launch_noise(o->seed, o->chain_id, T, D, f64, b + o_z, (double *)(b + o_u), st));
        xi = b + o_z;
        u = (const double *)(b + o_u);
    }
    PM_CUDA_R(rot_rows(b + o_xi, xi, tg->Q, T, D, true, f64, st));
    PM_CUDA_R(rot_rows(b + o_s0, s0, tg->Q, 1, D, true, f64, st));
    if (s_init) PM_CUDA_R(rot_rows(b + o_init, s_init, tg->Q, T, D, true, f64, st));
    pmcmc_target rt = *tg;
    rt.Q = nullptr;
    if (tg->kind == PMCMC_GAUSSIAN) {
        PM_CUDA_R(rot_rows(b + o_mu, tg->mean, tg->Q, 1, D, true, f64, st));
        PM_CUDA_R(rot_sym(b + o_P, tg->prec, tg->Q, D, f64, st));
        rt.mean = b + o_mu;
        rt.prec = b + o_P;
    } else {
        PM_CUDA_R(rot_rows(b + o_X, tg->X, tg->Q, tg->N, D, true, f64, st));  // rows X_n Q
        rt.X = b + o_X;
    }
    prof_count(c, 5);
    ps = newton_solve(c, &rt, o, T, b + o_s0, s_init ? b + o_init : nullptr, b + o_xi, u, b + o_z,
                      res, stream);
    if (ps < 0) return ps;
    PM_CUDA_R(rot_rows(s_out, b + o_z, tg->Q, T, D, false, f64, st));
    prof_count(c);
    PM_CUDA_R(cudaStreamSynchronize(st));
    return ps;
}

}  // namespace pm
