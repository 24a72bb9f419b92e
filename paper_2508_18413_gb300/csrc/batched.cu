// Batched solve of many independent chains of uneven T, D, sampler and target (the batching
// of Section 5.2: independent chains on one GPU) in one persistent launch.
//
// One cooperative kernel owns the whole GPU.  Each Newton sweep is a list of work items
// (chain c, tile k) over the chains that have not converged; CTAs take items in ticket order.
// An item evaluates and linearises the tile's timesteps (per-thread programs for Gaussian and
// banana targets, the shared-memory tile program for logistic regression), keeps the affine
// pairs (J_t, r_t) in shared memory, scans the tile, looks back along its chain for the carry
// (decoupled look-back, bounded waits), and writes s^(i+1) = s^(i) + delta into the chain's
// other ping-pong buffer, so no pair ever goes through HBM.  Between sweeps a bounded grid
// barrier lets CTA 0 apply Algorithm 1's stopping rule per chain
// (max |s^(i+1) - s^(i)| - rtol |s^(i+1)| <= atol) and build the next item list.
//
// Jacobians: MALA uses the exact diagonal (Eq. 4); HMC uses the diagonal of the tangent
// propagated with the diagonal of the Hessian (exact when H is diagonal; any diagonal keeps
// the fixed point).  FP32 arithmetic; with PMCMC_F32_SCAN_BF16 the pairs and the look-back
// aggregates are rounded to bfloat16 and combined in FP32.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "eval_small.cuh"
#include "logreg_tile.cuh"
#include "seq.h"
#include "solve.h"

namespace pm {

namespace {

constexpr int kBT = 256;          // threads per CTA
constexpr int kMaxTileSmall = 256;  // timesteps per item, per-thread programs

struct BChain {
    int target, sampler, D, T, L, N, DP;
    int tile_t, ntiles;
    float eps, sigma_p;
    const float *mu, *P, *Xp, *y, *s0, *xi;
    const double *u;
    float *buf0, *buf1;
    unsigned int *flags;
    float *agg, *incl;
};

struct BState {
    int iters, converged, parity, done;
    unsigned long long err;     // ord-encoded step-rule value of the current sweep
    unsigned long long resets;
    unsigned long long accepts;
    unsigned long long min_margin;
};

struct BCtl {
    unsigned int bar_count, bar_gen;
    unsigned int ticket, nitems;
    unsigned int epoch;
    unsigned int error;
    unsigned int sweeps, pad;
};

struct BArgs {
    int B;
    BChain *chains;
    BState *state;
    BCtl *ctl;
    int *active;
    unsigned int *prefix;
    int max_iters;  // <= 0: each chain's T
    double atol, rtol;
    float damping;
    int clip, bf16, gate_grad;
    unsigned int spin_limit;
};

__device__ __forceinline__ float bpost(float v, float damping, int clip) {
    v *= damping;
    if (clip) v = v > 1.f ? 1.f : (v < -1.f ? -1.f : v);
    return v;
}

__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Bounded grid barrier (all CTAs are co-resident: cooperative launch).
__device__ bool grid_barrier(BCtl *ctl, unsigned int nblocks, unsigned int limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned int gen = ld_acquire(&ctl->bar_gen);
        __threadfence();
        if (atomicAdd(&ctl->bar_count, 1u) == nblocks - 1) {
            ctl->bar_count = 0;
            __threadfence();
            st_release(&ctl->bar_gen, gen + 1);
        } else {
            Spin spin(limit);
            while (ld_acquire(&ctl->bar_gen) == gen) {
                if (!spin.again()) {
                    atomicExch(&ctl->error, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// ------------------------------------------------------------------------------------------
// Scan of one tile whose pairs sit in shared memory (Js, Rs: TTv x D, row-major), with the
// decoupled look-back along chain c; writes the new iterate and accumulates the step rule.
// ------------------------------------------------------------------------------------------
__device__ void tile_scan(const BChain &ch, BState *st, int k, int TTv, const float *Js,
                          const float *Rs, const float *sold, float *snew, float *segA,
                          float *segB, float *carry, unsigned int epoch, const BArgs &A,
                          BCtl *ctl) {
    const int D = ch.D, tid = threadIdx.x;
    const int NS = max(1, kBT / D);
    const int klen = ceil_div(TTv, NS);
    const int j = tid / D, d = tid - (tid / D) * D;
    const bool active = j < NS;
    const int i0 = j * klen, i1 = min(i0 + klen, TTv);
    float Aa = 1.f, Bb = 0.f;
    if (active)
        for (int i = i0; i < i1; i++) {
            const float ai = Js[i * D + d];
            Bb = ai * Bb + Rs[i * D + d];
            Aa = ai * Aa;
        }
    for (int off = 1; off < NS; off <<= 1) {
        if (active) {
            segA[tid] = Aa;
            segB[tid] = Bb;
        }
        __syncthreads();
        if (active && j >= off) {
            const float pa = segA[tid - off * D], pb = segB[tid - off * D];
            Bb = Aa * pb + Bb;
            Aa = Aa * pa;
        }
        __syncthreads();
    }
    if (active) {
        segA[tid] = Aa;
        segB[tid] = Bb;
    }
    __syncthreads();
    const int last = (NS - 1) * D;
    const unsigned int ep = epoch & 0x3fffffffu;
    if (tid < D) {
        float TA = segA[last + tid], TB = segB[last + tid];
        if (A.bf16) {
            TA = round_bf16(TA);
            TB = round_bf16(TB);
        }
        if (k == 0) {
            ch.incl[tid] = TB;
        } else {
            ch.agg[(size_t)k * 2 * D + tid] = TA;
            ch.agg[(size_t)k * 2 * D + D + tid] = TB;
        }
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) st_release(ch.flags + k, (ep << 2) | (k == 0 ? 2u : 1u));
    if (k > 0 && tid < D) {
        int jj = k - 1;
        bool timed_out = false;
        for (; jj >= 0; jj--) {
            Spin spin(A.spin_limit);
            unsigned int f;
            for (;;) {
                f = ld_acquire(ch.flags + jj);
                if ((f >> 2) == ep && (f & 3u)) break;
                if (!spin.again()) {
                    atomicExch(&ctl->error, 2u);
                    timed_out = true;
                    break;
                }
            }
            if (timed_out || (f & 3u) == 2u) break;
        }
        float c = 0.f;
        if (!timed_out && jj >= 0) c = ch.incl[(size_t)jj * D + tid];
        for (int m = max(jj + 1, 0); m < k; m++)
            c = ch.agg[(size_t)m * 2 * D + tid] * c + ch.agg[(size_t)m * 2 * D + D + tid];
        carry[tid] = c;
        float incl = segA[last + tid] * c + segB[last + tid];
        if (A.bf16) incl = round_bf16(incl);
        ch.incl[(size_t)k * D + tid] = incl;
        __threadfence();
    } else if (k == 0 && tid < D) {
        carry[tid] = 0.f;
    }
    __syncthreads();
    if (k > 0 && tid == 0) st_release(ch.flags + k, (ep << 2) | 2u);
    double err = -INFINITY;
    unsigned int resets = 0;
    if (active && i0 < i1) {
        float delta = carry[d];
        if (j > 0) delta = segA[tid - D] * delta + segB[tid - D];
        const size_t base = (size_t)0;
        (void)base;
        for (int i = i0; i < i1; i++) {
            delta = Js[i * D + d] * delta + Rs[i * D + d];
            const size_t o = (size_t)(k * ch.tile_t + i) * D + d;
            float sn = sold[o] + delta;
            if (!isfinite(sn)) {
                sn = ch.s0[d];
                resets++;
                err = INFINITY;
            } else {
                err = max(err, (double)fabsf(delta) - A.rtol * (double)fabsf(sn));
            }
            snew[o] = sn;
        }
    }
    err = warp_max(err);
    resets = warp_sum(resets);
    if ((tid & 31) == 0) {
        if (err > -INFINITY) atomic_max_d(&st->err, err);
        if (resets) atomicAdd(&st->resets, (unsigned long long)resets);
    }
}

// ------------------------------------------------------------------------------------------
// Per-thread programs (Gaussian, banana): thread tl evaluates timestep t0 + tl.
// ------------------------------------------------------------------------------------------
template <int DM, int TGT>
__device__ void eval_small_item(const BChain &ch, int t0, int TTv, const float *sold, float *Js,
                                float *Rs, float *smu, float *sP, const BArgs &A, BState *st) {
    const int D = ch.D, tl = threadIdx.x;
    using TG = typename TargetSel<float, DM, TGT>::type;
    TG tg;
    if constexpr (TGT == PMCMC_GAUSSIAN) {
        tg.mu = smu;
        tg.P = sP;
    }
    int acc_i = 0;
    double margin = INFINITY;
    if (tl < TTv) {
        const int t = t0 + tl;
        const float eps = ch.eps;
        const float *prev = t == 0 ? ch.s0 : sold + (size_t)(t - 1) * D;
        float x[DM], xi[DM], xc[DM], f[DM], jd[DM];
#pragma unroll
        for (int d = 0; d < DM; d++) {
            x[d] = d < D ? prev[d] : 0.f;
            xi[d] = d < D ? ch.xi[(size_t)t * D + d] : 0.f;
            xc[d] = d < D ? sold[(size_t)t * D + d] : 0.f;
        }
        const double u = ch.u[t];
        if (ch.sampler == PMCMC_MALA) {
            MalaState<float, DM, TG> m;
            mala_forward<float, DM>(tg, eps, x, xi, u, A.gate_grad != 0, m);
            acc_i = m.acc;
            margin = fabs(m.gtl);
            const float ga = m.acc ? 1.f : 0.f;
#pragma unroll
            for (int d = 0; d < DM; d++) {
                f[d] = m.acc ? m.xt[d] : m.x[d];
                jd[d] = ga * (1.f + eps * tg.hess(m.x, d, d)) + (1.f - ga) +
                        m.cg * (m.xt[d] - m.x[d]) * m.gl[d];
            }
        } else {
            HmcState<float, DM> h;
            hmc_forward<float, DM>(tg, eps, ch.L, x, xi, u, A.gate_grad != 0, h);
            acc_i = h.acc;
            margin = fabs(h.gtl);
            // diagonal tangent through the leapfrog with the Hessian diagonal
            float X[DM], V[DM], G[DM], dX[DM], dV[DM];
            const float he = 0.5f * eps;
#pragma unroll
            for (int d = 0; d < DM; d++) {
                X[d] = h.x0[d];
                V[d] = xi[d] + he * h.g0[d];
                G[d] = h.g0[d];
                dX[d] = 1.f;
                dV[d] = he * tg.hess(h.x0, d, d);
            }
            for (int l = 0; l < ch.L; l++) {
#pragma unroll
                for (int d = 0; d < DM; d++) {
                    X[d] += eps * V[d];
                    dX[d] += eps * dV[d];
                }
                tg.grad(X, G);
#pragma unroll
                for (int d = 0; d < DM; d++) {
                    V[d] += eps * G[d];
                    dV[d] += eps * tg.hess(X, d, d) * dX[d];
                }
            }
#pragma unroll
            for (int d = 0; d < DM; d++) {
                dV[d] -= he * tg.hess(X, d, d) * dX[d];
                V[d] -= he * G[d];
                f[d] = h.acc ? h.xL[d] : h.x0[d];
                const float dgt = -h.g0[d] - V[d] * dV[d] + G[d] * dX[d];
                jd[d] = (h.acc ? dX[d] : 1.f) + h.cg * (h.xL[d] - h.x0[d]) * dgt;
            }
        }
#pragma unroll
        for (int d = 0; d < DM; d++)
            if (d < D) {
                float jv = bpost(jd[d], A.damping, A.clip);
                float r = f[d] - xc[d];
                if (A.bf16) {
                    jv = round_bf16(jv);
                    r = round_bf16(r);
                }
                Js[tl * D + d] = jv;
                Rs[tl * D + d] = r;
            }
    }
    acc_i = __syncthreads_count(acc_i);
    margin = warp_min(margin);
    if ((threadIdx.x & 31) == 0 && margin < INFINITY) atomic_min_d(&st->min_margin, margin);
    if (threadIdx.x == 0 && acc_i) atomicAdd(&st->accepts, (unsigned long long)acc_i);
}

// ------------------------------------------------------------------------------------------
// Logistic-regression tile program (TT timesteps of one chain).
// ------------------------------------------------------------------------------------------
template <int DP>
__device__ void eval_logreg_item(const BChain &ch, int t0, int TTv, const float *sold, float *Js,
                                 float *Rs, unsigned char *smem, const BArgs &A, BState *st) {
    using namespace lr;
    using G = Geo<DP>;
    constexpr int TT = G::TT;
    Smem<float, DP> &S = *reinterpret_cast<Smem<float, DP> *>(smem);
    const int D = ch.D, N = ch.N, tid = threadIdx.x;
    const float eps = ch.eps, inv_sp2 = 1.f / (ch.sigma_p * ch.sigma_p);
    const int T = t0 + TTv;  // timesteps beyond the tile are masked
    for (int e = tid; e < TT * DP; e += kBT) {
        const int tl = e / DP, d = e - tl * DP;
        const int t = t0 + tl;
        float xp = 0.f, xv = 0.f, sv = 0.f;
        if (tl < TTv && d < D) {
            xp = t == 0 ? ch.s0[d] : sold[(size_t)(t - 1) * D + d];
            xv = ch.xi[(size_t)t * D + d];
            sv = sold[(size_t)t * D + d];
        }
        S.x[e] = xp;
        S.xi[e] = xv;
        S.sc[e] = sv;
        S.dh[e] = 0.f;
    }
    if (tid < TT) S.ll[tid] = 0.0;
    __syncthreads();
    int acc_i = 0;
    double margin = INFINITY;
    if (ch.sampler == PMCMC_MALA) {
        xpass<float, DP, kGrad>(S, ch.Xp, ch.y, N, S.x, nullptr, S.g, true, true, nullptr, t0, T);
        if (tid < TT) {
            S.ell[tid] = S.ll[tid];
            S.ll[tid] = 0.0;
        }
        const float sq = sqrtf(2.f * eps);
        for (int e = tid; e < TT * DP; e += kBT) {
            S.g[e] -= S.x[e] * inv_sp2;
            S.xt[e] = S.x[e] + eps * S.g[e] + sq * S.xi[e];
        }
        __syncthreads();
        xpass<float, DP, kGrad>(S, ch.Xp, ch.y, N, S.xt, nullptr, S.gt, true, false, nullptr, t0, T);
        for (int e = tid; e < TT * DP; e += kBT) {
            S.gt[e] -= S.xt[e] * inv_sp2;
            S.e[e] = S.x[e] - S.xt[e] - eps * S.gt[e];
        }
        __syncthreads();
        per_t_sum<float, DP>(TT, [&](int t, int d) {
            const int q = t * DP + d;
            const double xt = S.xt[q], x = S.x[q], e = S.e[q], xi = S.xi[q];
            return -(xt * xt - x * x) * 0.5 * (double)inv_sp2 - e * e / (4.0 * (double)eps) + 0.5 * xi * xi;
        }, S.gtl);
        __syncthreads();
        int any_gate = 0;
        if (tid < TT) {
            const double ell = (S.ll[tid] - S.ell[tid]) + S.gtl[tid];
            const int t = t0 + tid;
            const double u = tid < TTv ? ch.u[t] : 0.5;
            const double la = (ell < 0.0 || isnan(ell)) ? ell : 0.0;
            const double gtl = la - log(u);
            S.acc[tid] = (tid < TTv) && gtl > 0.0;
            S.cg[tid] = 0.f;
            if (A.gate_grad && ell < 0.0 && tid < TTv) {
                const double sg = 1.0 / (1.0 + exp(-gtl));
                S.cg[tid] = (float)(sg * (1.0 - sg));
                any_gate = 1;
            }
            if (tid < TTv) {
                acc_i = S.acc[tid];
                margin = fabs(gtl);
            }
        }
        any_gate = __syncthreads_or(any_gate);
        if (any_gate) {
            xpass<float, DP, kHvp>(S, ch.Xp, ch.y, N, S.xt, S.e, S.v, false, false, nullptr, t0, T);
            const float inv2e = 1.f / (2.f * eps);
            for (int e = tid; e < TT * DP; e += kBT) {
                const float He = -S.v[e] - S.e[e] * inv_sp2;
                S.v[e] = S.gt[e] + (S.e[e] + eps * He) * inv2e;
            }
            __syncthreads();
            xpass<float, DP, kHvp>(S, ch.Xp, ch.y, N, S.x, S.v, S.gl, false, false, nullptr, t0, T);
            for (int e = tid; e < TT * DP; e += kBT) {
                const float Hv = -S.gl[e] - S.v[e] * inv_sp2;
                S.gl[e] = S.v[e] + eps * Hv - S.g[e] - S.e[e] * inv2e;
            }
            __syncthreads();
        } else {
            for (int e = tid; e < TT * DP; e += kBT) S.gl[e] = 0.f;
            __syncthreads();
        }
        for (int e = tid; e < TTv * D; e += kBT) {
            const int tl = e / D, d = e - tl * D;
            const int q = tl * DP + d;
            const bool acc = S.acc[tl];
            const float f = acc ? S.xt[q] : S.x[q];
            const float ga = acc ? 1.f : 0.f;
            const float Hdd = -S.dh[q] - inv_sp2;
            float jv = bpost(ga * (1.f + eps * Hdd) + (1.f - ga) + S.cg[tl] * (S.xt[q] - S.x[q]) * S.gl[q],
                             A.damping, A.clip);
            float r = f - S.sc[q];
            if (A.bf16) {
                jv = round_bf16(jv);
                r = round_bf16(r);
            }
            Js[e] = jv;
            Rs[e] = r;
        }
    } else {
        // HMC: v0 = xi, half step, L leapfrogs, negative half step; diagonal tangent
        xpass<float, DP, kGrad>(S, ch.Xp, ch.y, N, S.x, nullptr, S.g, true, true, nullptr, t0, T);
        // S.g: grad at x0 (before prior), S.dh: diag X^T W X at x0, S.ll: loglik at x0
        if (tid < TT) {
            S.ell[tid] = S.ll[tid];  // ll(x0)
            S.ll[tid] = 0.0;
        }
        const float he = 0.5f * eps;
        for (int e = tid; e < TT * DP; e += kBT) {
            S.g[e] -= S.x[e] * inv_sp2;             // g0
            S.xt[e] = S.x[e];                       // X (position)
            S.v[e] = S.xi[e] + he * S.g[e];         // V
            S.e[e] = 1.f;                           // dX
            S.gl[e] = he * (-S.dh[e] - inv_sp2);    // dV
            S.gt[e] = S.g[e];                       // G
        }
        __syncthreads();
        for (int l = 0; l < ch.L; l++) {
            for (int e = tid; e < TT * DP; e += kBT) {
                S.xt[e] += eps * S.v[e];
                S.e[e] += eps * S.gl[e];
                S.dh[e] = 0.f;
            }
            if (tid < TT) S.ll[tid] = 0.0;
            __syncthreads();
            xpass<float, DP, kGrad>(S, ch.Xp, ch.y, N, S.xt, nullptr, S.gt, l == ch.L - 1, true,
                                    nullptr, t0, T);
            for (int e = tid; e < TT * DP; e += kBT) {
                S.gt[e] -= S.xt[e] * inv_sp2;
                S.v[e] += eps * S.gt[e];
                S.gl[e] += eps * (-S.dh[e] - inv_sp2) * S.e[e];
            }
            __syncthreads();
        }
        // negative half step; the Hessian diagonal at x_L is in dh
        for (int e = tid; e < TT * DP; e += kBT) {
            S.gl[e] -= he * (-S.dh[e] - inv_sp2) * S.e[e];
            S.v[e] -= he * S.gt[e];
        }
        __syncthreads();
        // H0 - HL = [|xi|^2/2 - lp(x0)] - [|vL|^2/2 - lp(xL)], lp = ll - |x|^2 / (2 sp^2)
        per_t_sum<float, DP>(TT, [&](int t, int d) {
            const int q = t * DP + d;
            const double xi = S.xi[q], v = S.v[q], x0 = S.x[q], xl = S.xt[q];
            return 0.5 * xi * xi - 0.5 * v * v + 0.5 * (double)inv_sp2 * (x0 * x0 - xl * xl);
        }, S.gtl);
        __syncthreads();
        if (tid < TT) {
            const double diff = S.gtl[tid] - S.ell[tid] + S.ll[tid];
            const int t = t0 + tid;
            const double u = tid < TTv ? ch.u[t] : 0.5;
            const double la = (diff < 0.0 || isnan(diff)) ? diff : 0.0;
            const double gtl = la - log(u);
            S.acc[tid] = (tid < TTv) && gtl > 0.0;
            S.cg[tid] = 0.f;
            if (A.gate_grad && diff < 0.0 && tid < TTv) {
                const double sg = 1.0 / (1.0 + exp(-gtl));
                S.cg[tid] = (float)(sg * (1.0 - sg));
            }
            if (tid < TTv) {
                acc_i = S.acc[tid];
                margin = fabs(gtl);
            }
        }
        __syncthreads();
        for (int e = tid; e < TTv * D; e += kBT) {
            const int tl = e / D, d = e - tl * D;
            const int q = tl * DP + d;
            const bool acc = S.acc[tl];
            const float f = acc ? S.xt[q] : S.x[q];
            const float dgt = -S.g[q] - S.v[q] * S.gl[q] + S.gt[q] * S.e[q];
            float jv = bpost((acc ? S.e[q] : 1.f) + S.cg[tl] * (S.xt[q] - S.x[q]) * dgt, A.damping,
                             A.clip);
            float r = f - S.sc[q];
            if (A.bf16) {
                jv = round_bf16(jv);
                r = round_bf16(r);
            }
            Js[e] = jv;
            Rs[e] = r;
        }
    }
    acc_i = __syncthreads_count(acc_i);
    margin = warp_min(margin);
    if ((tid & 31) == 0 && margin < INFINITY) atomic_min_d(&st->min_margin, margin);
    if (tid == 0 && acc_i) atomicAdd(&st->accepts, (unsigned long long)acc_i);
}

constexpr size_t kLogregSmem = sizeof(lr::Smem<float, 32>);
constexpr size_t kSmallSmem = 2 * sizeof(float) * kMaxTileSmall * 32 + sizeof(float) * (32 * 32 + 32);
constexpr size_t kEvalSmem = (kLogregSmem > kSmallSmem ? kLogregSmem : kSmallSmem);
constexpr size_t kPairSmem = 2 * sizeof(float) * 32 * 32;  // logistic tiles: TT x D pairs
constexpr size_t kScanSmem = sizeof(float) * (2 * kBT + 32);

}  // namespace

__global__ void __launch_bounds__(kBT) batched_kernel(BArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_item, s_epoch, s_nitems, s_stop, s_nact;
    __shared__ int s_chain;
    BCtl *ctl = A.ctl;
    const unsigned int nblocks = gridDim.x;
    unsigned char *eval_area = smem;
    float *pairs = reinterpret_cast<float *>(smem + kEvalSmem);
    float *scan_area = reinterpret_cast<float *>(smem + kEvalSmem + kPairSmem);
    float *segA = scan_area, *segB = scan_area + kBT, *carry = scan_area + 2 * kBT;
    for (int sweep = 0;; sweep++) {
        // CTA 0: stopping rule for the chains of the previous sweep, next item list
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) {
                unsigned int total = 0;
                int na = 0;
                for (int c = 0; c < A.B; c++) {
                    BState &s = A.state[c];
                    if (s.done) continue;
                    if (sweep > 0) {
                        s.iters++;
                        s.parity ^= 1;
                        const double err = ord_decode(s.err);
                        const int cap = A.max_iters > 0 ? A.max_iters : A.chains[c].T;
                        if (err <= A.atol) {
                            s.converged = 1;
                            s.done = 1;
                        } else if (s.iters >= cap) {
                            s.done = 1;
                        }
                    }
                    if (s.done) continue;
                    s.err = kOrdNegInf;
                    s.accepts = 0;
                    s.min_margin = 0xfff0000000000000ull;
                    A.active[na] = c;
                    A.prefix[na] = total;
                    total += A.chains[c].ntiles;
                    na++;
                }
                A.prefix[na] = total;
                ctl->pad = (unsigned int)na;
                ctl->nitems = total;
                ctl->ticket = 0;
                ctl->epoch = ctl->epoch + 1u;
                ctl->sweeps = sweep;
                __threadfence();
            }
        }
        if (!grid_barrier(ctl, nblocks, A.spin_limit)) return;
        if (threadIdx.x == 0) {
            s_nitems = *(volatile unsigned int *)&ctl->nitems;
            s_nact = *(volatile unsigned int *)&ctl->pad;
            s_epoch = *(volatile unsigned int *)&ctl->epoch;
            s_stop = (s_nitems == 0 || *(volatile unsigned int *)&ctl->error) ? 1u : 0u;
        }
        __syncthreads();
        if (s_stop) break;
        const unsigned int nitems = s_nitems, epoch = s_epoch;
        for (;;) {
            if (threadIdx.x == 0) {
                s_item = atomicAdd(&ctl->ticket, 1u);
                if (s_item < nitems) {
                    // active chain of this item: prefix[lo] <= item < prefix[lo + 1]
                    int lo = 0, hi = (int)s_nact;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (A.prefix[mid] <= s_item) lo = mid; else hi = mid;
                    }
                    s_chain = lo;
                }
            }
            __syncthreads();
            const unsigned int item = s_item;
            if (item >= nitems) break;
            const int ai = s_chain;
            const int c = A.active[ai];
            const BChain &ch = A.chains[c];
            BState *st = &A.state[c];
            const int k = (int)(item - A.prefix[ai]);
            const int t0 = k * ch.tile_t;
            const int TTv = min(ch.tile_t, ch.T - t0);
            const int par = st->parity;
            const float *sold = par ? ch.buf1 : ch.buf0;
            float *snew = par ? ch.buf0 : ch.buf1;
            float *Js = pairs, *Rs = pairs + 32 * 32;
            if (ch.target == PMCMC_LOGREG) {
                if (ch.DP == 16)
                    eval_logreg_item<16>(ch, t0, TTv, sold, Js, Rs, eval_area, A, st);
                else
                    eval_logreg_item<32>(ch, t0, TTv, sold, Js, Rs, eval_area, A, st);
            } else {
                float *sJ = reinterpret_cast<float *>(eval_area);
                float *sR = sJ + kMaxTileSmall * 32;
                float *sP = sR + kMaxTileSmall * 32;
                float *smu = sP + 32 * 32;
                Js = sJ;
                Rs = sR;
                if (ch.target == PMCMC_GAUSSIAN) {
                    const int DMp = ch.D <= 2 ? 2 : (ch.D <= 8 ? 8 : 32);
                    for (int e = threadIdx.x; e < DMp * DMp; e += kBT) {
                        const int i = e / DMp, jj = e % DMp;
                        sP[e] = (i < ch.D && jj < ch.D) ? ch.P[i * ch.D + jj] : 0.f;
                    }
                    for (int d = threadIdx.x; d < DMp; d += kBT) smu[d] = d < ch.D ? ch.mu[d] : 0.f;
                    __syncthreads();
                    if (DMp == 2)
                        eval_small_item<2, PMCMC_GAUSSIAN>(ch, t0, TTv, sold, Js, Rs, smu, sP, A, st);
                    else if (DMp == 8)
                        eval_small_item<8, PMCMC_GAUSSIAN>(ch, t0, TTv, sold, Js, Rs, smu, sP, A, st);
                    else
                        eval_small_item<32, PMCMC_GAUSSIAN>(ch, t0, TTv, sold, Js, Rs, smu, sP, A, st);
                } else {
                    eval_small_item<2, PMCMC_BANANA>(ch, t0, TTv, sold, Js, Rs, smu, sP, A, st);
                }
            }
            __syncthreads();
            tile_scan(ch, st, k, TTv, Js, Rs, sold, snew, segA, segB, carry, epoch, A, ctl);
            __syncthreads();
        }
        if (!grid_barrier(ctl, nblocks, A.spin_limit)) return;
    }
    // results: iterates held in buf1 go back to the caller's buffer
    for (int c = 0; c < A.B; c++) {
        const BChain &ch = A.chains[c];
        if (A.state[c].parity == 0) continue;
        const size_t n = (size_t)ch.T * ch.D;
        for (size_t i = (size_t)blockIdx.x * kBT + threadIdx.x; i < n; i += (size_t)gridDim.x * kBT)
            ch.buf0[i] = ch.buf1[i];
    }
}

__global__ void batched_init_kernel(BChain *chains, BState *state, int B) {
    const int c = blockIdx.x;
    if (c >= B) return;
    const BChain &ch = chains[c];
    const size_t n = (size_t)ch.T * ch.D;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) ch.buf0[i] = ch.s0[i % ch.D];
    if (threadIdx.x == 0) {
        BState &s = state[c];
        s.iters = 0;
        s.converged = 0;
        s.parity = 0;
        s.done = 0;
        s.err = kOrdNegInf;
        s.resets = 0;
        s.accepts = 0;
        s.min_margin = 0xfff0000000000000ull;
    }
}

}  // namespace pm

using namespace pm;

#define PM_CUDA_B(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return set_error(c, PMCMC_ECUDA, cudaGetErrorString(e_));      \
    } while (0)

namespace pm {

// Tile shapes of the batched kernel, chosen per workload signature by a small autotuner.
struct BatchTune {
    int small_tile = 256;  // timesteps per item, per-thread programs
    int blocks_per_sm = 0; // 0: occupancy maximum
};

static std::string tune_key(int B, const pmcmc_chain_desc *ch) {
    long long sumT = 0;
    int nl = 0, nh = 0, dmax = 0;
    for (int i = 0; i < B; i++) {
        sumT += ch[i].T;
        nl += ch[i].target.kind == PMCMC_LOGREG;
        nh += ch[i].sampler == PMCMC_HMC;
        dmax = std::max(dmax, ch[i].target.D);
    }
    char buf[160];
    snprintf(buf, sizeof(buf), "B%d_T%lld_lr%d_hmc%d_D%d", B, sumT, nl, nh, dmax);
    return buf;
}

}  // namespace pm

static pmcmc_status run_batched(pmcmc_ctx *c, int B, const pmcmc_chain_desc *chains,
                                const pmcmc_options *o, pmcmc_result *res, cudaStream_t st,
                                const BatchTune &tune, float *elapsed_ms, bool fill_results) {
    // workspace: descriptors, state, control, active list, prefix, per-chain buffers
    std::vector<BChain> hc(B);
    Carve cv;
    const size_t o_chains = cv.take(sizeof(BChain) * B);
    const size_t o_state = cv.take(sizeof(BState) * B);
    const size_t o_ctl = cv.take(sizeof(BCtl));
    const size_t o_active = cv.take(sizeof(int) * B);
    const size_t o_prefix = cv.take(sizeof(unsigned int) * (B + 1));
    std::vector<size_t> o_buf1(B), o_flags(B), o_agg(B), o_incl(B), o_xp(B);
    for (int i = 0; i < B; i++) {
        const pmcmc_chain_desc &d = chains[i];
        const int D = d.target.D;
        int tile = tune.small_tile;
        int DP = 0;
        if (d.target.kind == PMCMC_LOGREG) {
            DP = logreg_padded_dim(D);
            tile = lr::Geo<32>::TT;  // 32 for DP <= 32
        }
        const int nt = ceil_div(d.T, tile);
        o_buf1[i] = cv.take(sizeof(float) * (size_t)d.T * D);
        o_flags[i] = cv.take(sizeof(unsigned int) * nt);
        o_agg[i] = cv.take(sizeof(float) * (size_t)nt * 2 * D);
        o_incl[i] = cv.take(sizeof(float) * (size_t)nt * D);
        o_xp[i] = d.target.kind == PMCMC_LOGREG
                      ? cv.take(sizeof(float) * (size_t)ceil_div(d.target.N, 64) * 64 * DP)
                      : 0;
        BChain &b = hc[i];
        b.target = d.target.kind;
        b.sampler = d.sampler;
        b.D = D;
        b.T = d.T;
        b.L = d.leapfrog_L;
        b.N = d.target.N;
        b.DP = DP;
        b.tile_t = tile;
        b.ntiles = nt;
        b.eps = (float)d.step;
        b.sigma_p = (float)(d.target.prior_scale > 0 ? d.target.prior_scale : 1.0);
        b.mu = (const float *)d.target.mean;
        b.P = (const float *)d.target.prec;
        b.y = (const float *)d.target.y;
        b.s0 = (const float *)d.s0;
        b.xi = (const float *)d.xi;
        b.u = d.u;
        b.buf0 = (float *)d.s_out;
    }
    pmcmc_status ps = ws_reserve(c, cv.used);
    if (ps != PMCMC_OK) return ps;
    char *base = (char *)c->ws;
    for (int i = 0; i < B; i++) {
        BChain &b = hc[i];
        b.buf1 = (float *)(base + o_buf1[i]);
        b.flags = (unsigned int *)(base + o_flags[i]);
        b.agg = (float *)(base + o_agg[i]);
        b.incl = (float *)(base + o_incl[i]);
        b.Xp = b.target == PMCMC_LOGREG ? (const float *)(base + o_xp[i]) : nullptr;
        if (b.target == PMCMC_LOGREG) {
            const int Npad = ceil_div(b.N, 64) * 64;
            PM_CUDA_B(pad_rows_launch((void *)b.Xp, chains[i].target.X, b.N, b.D, Npad, b.DP, 4, st));
        }
        PM_CUDA_B(cudaMemsetAsync(b.flags, 0, sizeof(unsigned int) * b.ntiles, st));
    }
    c->flags_generation = ~0ull;
    BChain *dchains = (BChain *)(base + o_chains);
    BCtl *dctl = (BCtl *)(base + o_ctl);
    PM_CUDA_B(cudaMemcpyAsync(dchains, hc.data(), sizeof(BChain) * B, cudaMemcpyHostToDevice, st));
    PM_CUDA_B(cudaMemsetAsync(dctl, 0, sizeof(BCtl), st));
    batched_init_kernel<<<B, 256, 0, st>>>(dchains, (BState *)(base + o_state), B);
    PM_CUDA_B(cudaGetLastError());
    prof_count(c, 2);

    BArgs A;
    A.B = B;
    A.chains = dchains;
    A.state = (BState *)(base + o_state);
    A.ctl = dctl;
    A.active = (int *)(base + o_active);
    A.prefix = (unsigned int *)(base + o_prefix);
    A.max_iters = o->max_iters;
    A.atol = o->atol;
    A.rtol = o->rtol;
    A.damping = (float)(o->damping > 0 ? o->damping : 1.0);
    A.clip = o->clip;
    A.bf16 = o->precision == PMCMC_F32_SCAN_BF16;
    A.gate_grad = o->gate_grad;
    A.spin_limit = o->spin_limit > 0 ? (unsigned int)o->spin_limit : 1u << 26;

    const size_t smem = kEvalSmem + kPairSmem + kScanSmem;
    PM_CUDA_B(cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0, nsm = 0;
    PM_CUDA_B(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel, kBT, smem));
    PM_CUDA_B(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    if (occ < 1) return set_error(c, PMCMC_EUNSUPPORTED, "batched kernel does not fit on an SM");
    const int per_sm = tune.blocks_per_sm > 0 ? std::min(tune.blocks_per_sm, occ) : occ;
    const int grid = nsm * per_sm;

    // the persistent launch, captured once into a CUDA graph and replayed
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaEventRecord(c->ev0, st);
    prof_begin(c, 0, st);
    // capture the persistent launch into a CUDA graph once per (workspace, chains, shape) and
    // replay it; fall back to a direct launch if the capture is refused
    char key[128];
    snprintf(key, sizeof(key), "%llu:%d:%d:%d", c->ws_generation, B, grid, tune.small_tile);
    bool launched = false;
    if (c->batch_graph_key == key && c->batch_graph_exec) {
        launched = cudaGraphLaunch(c->batch_graph_exec, st) == cudaSuccess;
        if (!launched) cudaGetLastError();
    } else {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t le = cudaLaunchKernelEx(&cfg, batched_kernel, A);
            cudaError_t ce = cudaStreamEndCapture(st, &g);
            cudaGraphExec_t ge = nullptr;
            if (le == cudaSuccess && ce == cudaSuccess && g &&
                cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
                if (c->batch_graph_exec) cudaGraphExecDestroy(c->batch_graph_exec);
                c->batch_graph_exec = ge;
                c->batch_graph_key = key;
                launched = cudaGraphLaunch(ge, st) == cudaSuccess;
            }
            if (g) cudaGraphDestroy(g);
        }
        if (!launched) cudaGetLastError();
    }
    if (!launched) PM_CUDA_B(cudaLaunchKernelEx(&cfg, batched_kernel, A));
    prof_end(c, 0, st);
    prof_count(c, 1);
    cudaEventRecord(c->ev1, st);
    std::vector<BState> hs(B);
    BCtl hctl;
    PM_CUDA_B(cudaMemcpyAsync(hs.data(), A.state, sizeof(BState) * B, cudaMemcpyDeviceToHost, st));
    PM_CUDA_B(cudaMemcpyAsync(&hctl, dctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
    PM_CUDA_B(cudaStreamSynchronize(st));
    prof_collect(c, 0);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    if (elapsed_ms) *elapsed_ms = ms;
    if (hctl.error) return set_error(c, PMCMC_ETIMEOUT, "batched: a bounded device wait ran out");
    bool all = true;
    for (int i = 0; i < B; i++) {
        all = all && hs[i].converged;
        if (fill_results && res) {
            res[i].iters = hs[i].iters;
            res[i].status = hs[i].converged ? PMCMC_OK : PMCMC_NOT_CONVERGED;
            res[i].max_residual = ord_decode(hs[i].err);
            res[i].accept_rate = (double)hs[i].accepts / (double)chains[i].T;
            res[i].min_margin = ord_decode(hs[i].min_margin);
            res[i].nonfinite_resets = (int)hs[i].resets;
            res[i].elapsed_ms = ms;
        }
    }
    return all ? PMCMC_OK : PMCMC_NOT_CONVERGED;
}

namespace pm {
BatchTune batch_tune_lookup(pmcmc_ctx *c, int B, const pmcmc_chain_desc *chains,
                            const pmcmc_options *o, cudaStream_t st);
}

namespace pm {

static SeqChain seq_of(const pmcmc_chain_desc &d) {
    SeqChain q;
    q.target = d.target.kind;
    q.sampler = d.sampler;
    q.D = d.target.D;
    q.N = d.target.N;
    q.L = d.leapfrog_L;
    q.T = d.T;
    q.eps = d.step;
    q.sigma_p = d.target.prior_scale;
    q.X = d.target.X;
    q.y = d.target.y;
    q.mu = d.target.mean;
    q.P = d.target.prec;
    q.s0 = d.s0;
    q.xi = d.xi;
    q.u = d.u;
    q.s_out = d.s_out;
    return q;
}

// The sequential loops of the chains `idx` in one launch, one CTA per chain, the longest chains
// first (their CTAs are dispatched first when the chains outnumber the resident CTAs).
static cudaError_t seq_batch_launch(pmcmc_ctx *c, const pmcmc_chain_desc *ch, std::vector<int> idx,
                                    bool f64, cudaStream_t st) {
    if (idx.empty()) return cudaSuccess;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return ch[a].T > ch[b].T; });
    std::vector<SeqChain> v;
    size_t smem = 0;
    for (int i : idx) {
        v.push_back(seq_of(ch[i]));
        smem = std::max(smem, seq_smem_bytes(v.back(), 1, kSeqThreadsBatched, f64));
    }
    const size_t bytes = sizeof(SeqChain) * v.size();
    if (c->seq_desc_bytes < bytes) {
        if (c->seq_desc) {
            cudaError_t e = cudaStreamSynchronize(st);  // the old descriptors may still be read
            if (e != cudaSuccess) return e;
            cudaFree(c->seq_desc);
            c->seq_desc = nullptr;
            c->seq_desc_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&c->seq_desc, bytes);
        if (e != cudaSuccess) return e;
        c->seq_desc_bytes = bytes;
    }
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(c->seq_desc, v.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    prof_count(c);
    return launch_seq_chains(static_cast<const SeqChain *>(c->seq_desc), (int)v.size(), smem, f64, st);
}

static bool seq_batch_ok(const pmcmc_chain_desc &d, bool f64) {
    const SeqChain q = seq_of(d);
    return seq_fast_supported(q) && seq_smem_bytes(q, 1, kSeqThreadsBatched, f64) <= kSeqSmemBudget;
}

// Chains still unconverged after the Newton sweeps are recomputed by the sequential loop: all
// Gaussian and logistic chains in one launch, one CTA each; any other chain (banana) on the
// context's side streams, up to sixteen at once (ordered after `st`, and `st` after them).
static cudaError_t complete_sequential(pmcmc_ctx *c, int B, const pmcmc_chain_desc *ch,
                                       pmcmc_result *rv, cudaStream_t st) {
    std::vector<int> todo, batch;
    for (int i = 0; i < B; i++) {
        if (rv[i].status != PMCMC_NOT_CONVERGED) continue;
        rv[i].status = PMCMC_OK;
        rv[i].sequential = 1;
        rv[i].max_residual = 0.0;
        (seq_batch_ok(ch[i], false) ? batch : todo).push_back(i);
    }
    cudaError_t eb = seq_batch_launch(c, ch, batch, false, st);
    if (eb != cudaSuccess) return eb;
    if (todo.empty()) return cudaSuccess;
    for (cudaStream_t &q : c->seq_streams)
        if (!q) {
            cudaError_t e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
        }
    for (cudaEvent_t &ev : c->seq_events)
        if (!ev) {
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
    const int nq = std::min<int>(16, (int)todo.size());
    cudaError_t e = cudaEventRecord(c->seq_events[16], st);
    for (int k = 0; k < nq && e == cudaSuccess; k++) e = cudaStreamWaitEvent(c->seq_streams[k], c->seq_events[16], 0);
    if (e != cudaSuccess) return e;
    for (size_t j = 0; j < todo.size(); j++) {
        const int i = todo[j];
        const pmcmc_chain_desc &d = ch[i];
        pmcmc_options so;
        pmcmc_options_default(&so);
        so.sampler = d.sampler;
        so.step = d.step;
        so.leapfrog_L = d.leapfrog_L;
        so.precision = PMCMC_F32;
        EvalArgs A;
        fill_eval_args(A, &d.target, &so, d.T);
        A.s0 = d.s0;
        A.xi = d.xi;
        A.u = d.u;
        A.f_out = d.s_out;
        cudaStream_t q = c->seq_streams[j % nq];
        e = d.target.kind == PMCMC_LOGREG ? launch_seq_logreg(A, q) : launch_seq_small(A, q);
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k < nq && e == cudaSuccess; k++) {
        e = cudaEventRecord(c->seq_events[k], c->seq_streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->seq_events[k], 0);
    }
    return e;
}

}  // namespace pm

extern "C" pmcmc_status pmcmc_solve_batched(pmcmc_ctx *c, int B, const pmcmc_chain_desc *chains,
                                            const pmcmc_options *o, pmcmc_result *res,
                                            void *stream) {
    if (!c) return PMCMC_EINVAL;
    if (B < 0 || (B > 0 && !chains) || !o) return set_error(c, PMCMC_EINVAL, "batched: bad arguments");
    if (B == 0) return PMCMC_OK;
    if (o->precision == PMCMC_F64) return set_error(c, PMCMC_EUNSUPPORTED, "batched: FP32 precisions");
    if (o->jac != PMCMC_JAC_DIAG) return set_error(c, PMCMC_EUNSUPPORTED, "batched: DIAG Jacobian");
    for (int i = 0; i < B; i++) {
        const pmcmc_chain_desc &d = chains[i];
        const pmcmc_target &t = d.target;
        if (d.T < 1 || !d.s0 || !d.xi || !d.u || !d.s_out || !(d.step > 0))
            return set_error(c, PMCMC_EINVAL, "batched: chain with bad T, buffers or step");
        if (d.sampler != PMCMC_MALA && d.sampler != PMCMC_HMC)
            return set_error(c, PMCMC_EINVAL, "batched: MALA or HMC chains");
        if (d.sampler == PMCMC_HMC && d.leapfrog_L < 1) return set_error(c, PMCMC_EINVAL, "batched: HMC needs L >= 1");
        if (t.kind == PMCMC_GAUSSIAN) {
            if (t.D < 1 || t.D > 32 || !t.mean || !t.prec)
                return set_error(c, PMCMC_EINVAL, "batched: Gaussian chains need D <= 32, mean, prec");
        } else if (t.kind == PMCMC_LOGREG) {
            if (t.D < 1 || t.D > 32 || !t.X || !t.y || t.N < 1)
                return set_error(c, PMCMC_EINVAL, "batched: logistic chains need D <= 32, X, y");
        } else if (t.kind == PMCMC_BANANA) {
            if (t.D != 2) return set_error(c, PMCMC_EINVAL, "batched: banana has D = 2");
        } else {
            return set_error(c, PMCMC_EINVAL, "batched: unknown target");
        }
    }
    PM_CUDA_B(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    // chains with an orthogonal basis Q (Section 3.4) are solved in rotated coordinates
    bool any_q = false;
    for (int i = 0; i < B; i++) any_q = any_q || chains[i].target.Q;
    std::vector<pmcmc_chain_desc> rc;
    const pmcmc_chain_desc *use = chains;
    if (any_q) {
        rc.assign(chains, chains + B);
        Carve cv;
        std::vector<size_t> off(B);
        for (int i = 0; i < B; i++) {
            if (!chains[i].target.Q) continue;
            const pmcmc_chain_desc &d = chains[i];
            const int D = d.target.D;
            off[i] = cv.take(sizeof(float) * ((size_t)2 * d.T * D + 2 * D + (size_t)D * D +
                                              (d.target.kind == PMCMC_LOGREG ? (size_t)d.target.N * D : 0)));
        }
        pmcmc_status ps = aux_reserve(c, cv.used);
        if (ps != PMCMC_OK) return ps;
        for (int i = 0; i < B; i++) {
            if (!chains[i].target.Q) continue;
            const pmcmc_chain_desc &d = chains[i];
            const int D = d.target.D;
            float *p = (float *)((char *)c->aux + off[i]);
            float *xi = p, *z = xi + (size_t)d.T * D, *s0 = z + (size_t)d.T * D, *mu = s0 + D;
            float *P = mu + D, *X = P + (size_t)D * D;
            PM_CUDA_B(rot_rows(xi, d.xi, d.target.Q, d.T, D, true, false, st));
            PM_CUDA_B(rot_rows(s0, d.s0, d.target.Q, 1, D, true, false, st));
            pmcmc_chain_desc &r = rc[i];
            r.xi = xi;
            r.s0 = s0;
            r.s_out = z;
            r.target.Q = nullptr;
            if (d.target.kind == PMCMC_GAUSSIAN) {
                PM_CUDA_B(rot_rows(mu, d.target.mean, d.target.Q, 1, D, true, false, st));
                PM_CUDA_B(rot_sym(P, d.target.prec, d.target.Q, D, false, st));
                r.target.mean = mu;
                r.target.prec = P;
            } else if (d.target.kind == PMCMC_LOGREG) {
                PM_CUDA_B(rot_rows(X, d.target.X, d.target.Q, d.target.N, D, true, false, st));
                r.target.X = X;
            } else {
                return set_error(c, PMCMC_EUNSUPPORTED, "batched: basis Q for Gaussian or logistic chains");
            }
        }
        use = rc.data();
    }
    BatchTune tune = batch_tune_lookup(c, B, use, o, st);
    pmcmc_options ob = *o;
    if (o->seq_after > 0 && (o->max_iters <= 0 || o->seq_after < o->max_iters)) ob.max_iters = o->seq_after;
    std::vector<pmcmc_result> rv(B);
    pmcmc_status ps = run_batched(c, B, use, &ob, rv.data(), st, tune, nullptr, true);
    for (int i = 0; i < B; i++) rv[i].sequential = 0;
    if (o->seq_after > 0 && ps >= 0) {
        PM_CUDA_B(complete_sequential(c, B, use, rv.data(), st));
        ps = PMCMC_OK;
        for (int i = 0; i < B; i++)
            if (rv[i].status != PMCMC_OK) ps = (pmcmc_status)rv[i].status;
    }
    if (res) std::copy(rv.begin(), rv.end(), res);
    if (any_q && ps >= 0) {
        for (int i = 0; i < B; i++)
            if (chains[i].target.Q)
                PM_CUDA_B(rot_rows(chains[i].s_out, rc[i].s_out, chains[i].target.Q, chains[i].T,
                                   chains[i].target.D, false, false, st));
        PM_CUDA_B(cudaStreamSynchronize(st));
    }
    return ps;
}

namespace pm {

// Autotuner: for a new workload signature, time a few tile shapes on two Newton sweeps of the
// actual problem and keep the fastest (cached per context, and in the file named by
// PMCMC_TUNE_CACHE when that variable is set).
BatchTune batch_tune_lookup(pmcmc_ctx *c, int B, const pmcmc_chain_desc *chains,
                            const pmcmc_options *o, cudaStream_t st) {
    const std::string key = tune_key(B, chains);
    auto it = c->tune_cache.find(key);
    if (it != c->tune_cache.end()) {
        BatchTune t;
        t.small_tile = it->second.first;
        t.blocks_per_sm = it->second.second;
        return t;
    }
    const char *path = getenv("PMCMC_TUNE_CACHE");
    if (path) {
        FILE *f = fopen(path, "r");
        if (f) {
            char k[256];
            int a, b;
            while (fscanf(f, "%255s %d %d", k, &a, &b) == 3)
                if (key == k) {
                    fclose(f);
                    c->tune_cache[key] = {a, b};
                    BatchTune t;
                    t.small_tile = a;
                    t.blocks_per_sm = b;
                    return t;
                }
            fclose(f);
        }
    }
    pmcmc_options probe = *o;
    probe.max_iters = 2;
    BatchTune best;
    float best_ms = 1e30f;
    const int tiles[] = {64, 128, 256};
    const int occs[] = {0, 1, 2};
    for (int tt : tiles)
        for (int bs : occs) {
            BatchTune t;
            t.small_tile = tt;
            t.blocks_per_sm = bs;
            float ms = 0.f;
            const int saved = c->prof_on;
            c->prof_on = 0;
            pmcmc_status s = run_batched(c, B, chains, &probe, nullptr, st, t, &ms, false);
            c->prof_on = saved;
            if ((s == PMCMC_OK || s == PMCMC_NOT_CONVERGED) && ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    c->tune_cache[key] = {best.small_tile, best.blocks_per_sm};
    if (path) {
        FILE *f = fopen(path, "a");
        if (f) {
            fprintf(f, "%s %d %d\n", key.c_str(), best.small_tile, best.blocks_per_sm);
            fclose(f);
        }
    }
    return best;
}

}  // namespace pm

extern "C" pmcmc_status pmcmc_seq_solve_batched(pmcmc_ctx *c, int B, const pmcmc_chain_desc *chains,
                                                const pmcmc_options *o, void *stream) {
    using namespace pm;
    if (!c) return PMCMC_EINVAL;
    if (B < 0 || (B > 0 && !chains) || !o) return set_error(c, PMCMC_EINVAL, "seq batched: bad arguments");
    if (B == 0) return PMCMC_OK;
    if (o->precision != PMCMC_F32 && o->precision != PMCMC_F64)
        return set_error(c, PMCMC_EINVAL, "seq batched: F32 or F64");
    const bool f64 = o->precision == PMCMC_F64;
    std::vector<int> idx;
    for (int i = 0; i < B; i++) {
        const pmcmc_chain_desc &d = chains[i];
        const pmcmc_target &t = d.target;
        if (d.T < 1 || !d.s0 || !d.xi || !d.u || !d.s_out)
            return set_error(c, PMCMC_EINVAL, "seq batched: chain with bad T or buffers");
        if (d.sampler != PMCMC_MALA && d.sampler != PMCMC_HMC)
            return set_error(c, PMCMC_EINVAL, "seq batched: MALA or HMC chains");
        if (t.kind == PMCMC_GAUSSIAN ? (!t.mean || !t.prec) : (t.kind != PMCMC_LOGREG || !t.X || !t.y || t.N < 1))
            return set_error(c, PMCMC_EINVAL, "seq batched: Gaussian (mean, prec) or logistic (X, y) chains");
        if (!seq_batch_ok(d, f64))
            return set_error(c, PMCMC_EUNSUPPORTED, "seq batched: D <= 128 and the design in one SM's shared memory");
        idx.push_back(i);
    }
    PM_CUDA_B(cudaSetDevice(c->device));
    PM_CUDA_B(seq_batch_launch(c, chains, idx, f64, (cudaStream_t)stream));
    return PMCMC_OK;
}
