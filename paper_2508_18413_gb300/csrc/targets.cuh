// Per-thread target densities for small D (the state of one timestep lives in registers).
// log p is returned up to an additive constant, as the MH ratio needs only differences.
//   Gaussian:  log p = -1/2 (x - mu)^T P (x - mu),  grad = -P (x - mu),  H = -P
//   Banana:    log p = -x1^2/200 - b^2/2 with b = x2 + 0.1 x1^2 - 10 (D = 2)
// Arrays have the compile-time capacity DM; entries d >= D are zero and stay zero.
#pragma once

#include "common.cuh"

namespace pm {

template <typename R, int DM>
struct GaussianT {
    const R *mu;  // shared memory, DM
    const R *P;   // shared memory, DM x DM (zero padded)
    __device__ __forceinline__ void grad(const R *x, R *g) const {
        R xm[DM];
#pragma unroll
        for (int j = 0; j < DM; j++) xm[j] = x[j] - mu[j];
#pragma unroll
        for (int i = 0; i < DM; i++) {
            R acc = R(0);
#pragma unroll
            for (int j = 0; j < DM; j++) acc = fma(P[i * DM + j], xm[j], acc);
            g[i] = -acc;
        }
    }
    // log p from the gradient at the same point: 1/2 (x - mu) . g
    __device__ __forceinline__ double logp(const R *x, const R *g) const {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < DM; i++) acc += (double)(x[i] - mu[i]) * (double)g[i];
        return 0.5 * acc;
    }
    __device__ __forceinline__ void hvp(const R *x, const R *v, R *out) const {
        (void)x;
#pragma unroll
        for (int i = 0; i < DM; i++) {
            R acc = R(0);
#pragma unroll
            for (int j = 0; j < DM; j++) acc = fma(P[i * DM + j], v[j], acc);
            out[i] = -acc;
        }
    }
    __device__ __forceinline__ R hess(const R *x, int i, int j) const {
        (void)x;
        return -P[i * DM + j];
    }
};

template <typename R, int DM>
struct BananaT {
    static_assert(DM == 2, "banana target is two-dimensional");
    __device__ __forceinline__ void grad(const R *x, R *g) const {
        const R b = x[1] + R(0.1) * x[0] * x[0] - R(10);
        g[0] = -x[0] * R(0.01) - R(0.2) * x[0] * b;
        g[1] = -b;
    }
    __device__ __forceinline__ double logp(const R *x, const R *g) const {
        (void)g;
        const double x0 = x[0], x1 = x[1];
        const double b = x1 + 0.1 * x0 * x0 - 10.0;
        return -x0 * x0 / 200.0 - 0.5 * b * b;
    }
    __device__ __forceinline__ R hess(const R *x, int i, int j) const {
        const R b = x[1] + R(0.1) * x[0] * x[0] - R(10);
        if (i == 0 && j == 0) return R(-0.01) - R(0.04) * x[0] * x[0] - R(0.2) * b;
        if (i == 1 && j == 1) return R(-1);
        return R(-0.2) * x[0];
    }
    __device__ __forceinline__ void hvp(const R *x, const R *v, R *out) const {
        const R h00 = hess(x, 0, 0), h01 = R(-0.2) * x[0];
        out[0] = h00 * v[0] + h01 * v[1];
        out[1] = h01 * v[0] - v[1];
    }
};

}  // namespace pm
