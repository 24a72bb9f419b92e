// Shared-memory tile machinery of the logistic-regression passes: a CTA owns TT timesteps and
// streams the design matrix X through shared memory in sub-chunks of kNC rows, computing
//   Z = V X^T (TT x N),  an elementwise map,  G = C X (TT x D)
// for one or two state blocks V.  Used by the evaluate-and-linearise kernel and the batched
// persistent kernel.
#pragma once

#include "common.cuh"
#include "eval.h"

namespace pm {
namespace lr {

constexpr int kNT = 256;  // threads: ty = tid / 16 (timesteps), tx = tid % 16 (rows / columns)
constexpr int kNC = 64;   // X rows per sub-chunk

template <int DP>
struct Geo {
    static constexpr int TT = DP >= 64 ? 16 : 32;  // timesteps per CTA
    static constexpr int MT = TT / 16;             // timesteps per thread in the contractions
    static constexpr int NJ = kNC / 16;            // X rows per thread in Z = V X^T
    static constexpr int DJ = DP / 16;             // columns per thread in G = C X
    static constexpr int XS = DP + 1;              // shared row stride of the X sub-chunk
};

template <typename R>
__device__ __forceinline__ R sigm(R z) { return R(1) / (R(1) + exp(-z)); }

template <typename R>
__device__ __forceinline__ R softplus(R z) { return z > R(0) ? z + log1p(exp(-z)) : log1p(exp(z)); }

template <typename R>
__device__ __forceinline__ R post_j(R v, R damping, int clip) {
    v *= damping;
    if (clip) v = v > R(1) ? R(1) : (v < R(-1) ? R(-1) : v);
    return v;
}

enum PassMode { kGrad = 0, kHvp = 1 };

// Shared-memory layout of one CTA.
template <typename R, int DP>
struct Smem {
    using G = Geo<DP>;
    R Xs[kNC * G::XS];
    R Cs[G::TT * kNC];
    R Ws[G::TT * kNC];
    R x[G::TT * DP], xi[G::TT * DP], sc[G::TT * DP], xt[G::TT * DP];
    R g[G::TT * DP], gt[G::TT * DP], e[G::TT * DP], v[G::TT * DP];
    R dh[G::TT * DP], gl[G::TT * DP];
    R ys[kNC];
    double ll[G::TT];
    double ell[G::TT], gtl[G::TT];
    R cg[G::TT];
    int acc[G::TT];
};

// One pass over X for the CTA's TT states.
//   kGrad: out = X^T (y - sigmoid(V1 X^T)); ll[t] += sum_n y z - softplus(z) (if want_ll);
//          dh = X^T(w) X diag (if want_w); w per (t, n) to wout (if wout).
//   kHvp:  out = X^T (w(V1 X^T) (.) (V2 X^T)).
template <typename R, int DP, int MODE>
__device__ void xpass(Smem<R, DP> &S, const R *__restrict__ Xp, const R *__restrict__ y, int N,
                      const R *V1, const R *V2, R *out, bool want_ll, bool want_w, R *wout,
                      int t0, int T) {
    using G = Geo<DP>;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    R acc[G::MT][G::DJ], accw[G::MT][G::DJ];
    double llp[G::MT];  // FP64 sum over chunks of per-chunk partials (NC/16 terms each)
#pragma unroll
    for (int i = 0; i < G::MT; i++) {
        llp[i] = 0.0;
#pragma unroll
        for (int j = 0; j < G::DJ; j++) acc[i][j] = accw[i][j] = R(0);
    }
    const int nchunks = ceil_div(N, kNC);
    for (int c = 0; c < nchunks; c++) {
        const int n0 = c * kNC;
        __syncthreads();  // previous consumers of Xs / Cs are done
        for (int e = tid; e < kNC * DP; e += kNT) {
            const int r = e / DP, k = e - r * DP;
            S.Xs[r * G::XS + k] = Xp[(size_t)(n0 + r) * DP + k];  // Xp rows are padded to kNC
        }
        if (MODE == kGrad && tid < kNC) S.ys[tid] = (n0 + tid < N) ? y[n0 + tid] : R(0);
        __syncthreads();
        // Z = V1 X^T (and Q = V2 X^T for the Hessian-vector product)
        R z1[G::MT][G::NJ], z2[G::MT][G::NJ];
#pragma unroll
        for (int i = 0; i < G::MT; i++)
#pragma unroll
            for (int j = 0; j < G::NJ; j++) z1[i][j] = z2[i][j] = R(0);
#pragma unroll 4
        for (int k = 0; k < DP; k++) {
            R a1[G::MT], a2[G::MT], b[G::NJ];
#pragma unroll
            for (int i = 0; i < G::MT; i++) {
                a1[i] = V1[(ty + 16 * i) * DP + k];
                if (MODE == kHvp) a2[i] = V2[(ty + 16 * i) * DP + k];
            }
#pragma unroll
            for (int j = 0; j < G::NJ; j++) b[j] = S.Xs[(tx + 16 * j) * G::XS + k];
#pragma unroll
            for (int i = 0; i < G::MT; i++)
#pragma unroll
                for (int j = 0; j < G::NJ; j++) {
                    z1[i][j] = fma(a1[i], b[j], z1[i][j]);
                    if (MODE == kHvp) z2[i][j] = fma(a2[i], b[j], z2[i][j]);
                }
        }
        // elementwise map
#pragma unroll
        for (int i = 0; i < G::MT; i++) {
            const int tl = ty + 16 * i;
            R llc = R(0);
#pragma unroll
            for (int j = 0; j < G::NJ; j++) {
                const int nl = tx + 16 * j;
                const bool valid = n0 + nl < N;
                const R z = z1[i][j];
                const R p = sigm(z);
                const R w = p * (R(1) - p);
                if (MODE == kGrad) {
                    S.Cs[tl * kNC + nl] = valid ? S.ys[nl] - p : R(0);
                    if (want_w) S.Ws[tl * kNC + nl] = valid ? w : R(0);
                    if (want_ll && valid) llc += S.ys[nl] * z - softplus(z);
                    if (wout && valid && t0 + tl < T) wout[(size_t)(t0 + tl) * N + n0 + nl] = w;
                } else {
                    S.Cs[tl * kNC + nl] = valid ? w * z2[i][j] : R(0);
                }
            }
            if (MODE == kGrad && want_ll) llp[i] += (double)llc;
        }
        __syncthreads();
        // G += C X  (and diag(X^T W X) += W X^2)
#pragma unroll 4
        for (int n = 0; n < kNC; n++) {
            R cc[G::MT], ww[G::MT], xv[G::DJ];
#pragma unroll
            for (int i = 0; i < G::MT; i++) {
                cc[i] = S.Cs[(ty + 16 * i) * kNC + n];
                if (MODE == kGrad && want_w) ww[i] = S.Ws[(ty + 16 * i) * kNC + n];
            }
#pragma unroll
            for (int j = 0; j < G::DJ; j++) xv[j] = S.Xs[n * G::XS + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < G::MT; i++)
#pragma unroll
                for (int j = 0; j < G::DJ; j++) {
                    acc[i][j] = fma(cc[i], xv[j], acc[i][j]);
                    if (MODE == kGrad && want_w) accw[i][j] = fma(ww[i] * xv[j], xv[j], accw[i][j]);
                }
        }
    }
    // write results
#pragma unroll
    for (int i = 0; i < G::MT; i++) {
        const int tl = ty + 16 * i;
#pragma unroll
        for (int j = 0; j < G::DJ; j++) {
            out[tl * DP + tx + 16 * j] = acc[i][j];
            if (MODE == kGrad && want_w) S.dh[tl * DP + tx + 16 * j] = accw[i][j];
        }
        if (MODE == kGrad && want_ll) {
            double l = llp[i];
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
            if (tx == 0) S.ll[tl] += l;
        }
    }
    __syncthreads();
}

// Per-timestep reduction over the DP entries of a shared vector expression (warp per t).
template <typename R, int DP, class F>
__device__ __forceinline__ void per_t_sum(int TT, F f, double *dst) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = w; t < TT; t += kNT / 32) {
        double acc = 0.0;
        for (int d = lane; d < DP; d += 32) acc += f(t, d);
        acc = warp_sum(acc);
        if (lane == 0) dst[t] = acc;
    }
}


}  // namespace lr
}  // namespace pm
