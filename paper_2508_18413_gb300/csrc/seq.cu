// The sequential chain s_t = f_t(s_{t-1}) on the GPU: the baseline the parallel Newton solve is
// measured against (the paper's sequential loop, Section 5).  A baseline is only as honest as it
// is fast, so this loop is written for latency: one dependent step after another, each step as
// short as the device allows.
//
//   * One CTA (or a cluster of CTAs) per chain.  A logistic-regression target keeps its design
//     rows resident in shared memory (row stride D | 1, conflict-free for row dots and column
//     sums); a cluster of 2..16 CTAs splits the rows when they do not fit one SM, and the
//     per-CTA partial gradients and log-likelihoods are summed through distributed shared memory
//     in rank order, so every CTA of a cluster holds bit-identical sums and takes the same
//     accept decision.
//   * The gradient and log-density at the current state are carried from step to step (a
//     rejected step keeps them, an accepted one takes the proposal's), so a MALA step costs one
//     gradient evaluation and an HMC step L.
//   * The next step's noise is prefetched into registers during the current step.
// The arithmetic follows Section 3.2 (MALA: proposal, MH log-ratio with the proposal densities,
// strict acceptance log alpha - log u > 0) and Algorithm 2 (HMC with a sequential leapfrog,
// accept iff log u < H_0 - H_L); the log-ratio and the comparison are in FP64.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "eval.h"
#include "internal.h"
#include "seq.h"

namespace pm {

namespace cg = cooperative_groups;

namespace {

constexpr int kDMax = kSeqDMax;

struct SeqCtx {
    int target, sampler, D, N, L, T, Dp, rows, row0, K, cs, rank;
};

// Scratch doubles at the start of dynamic shared memory (then the R arrays).
constexpr int kRed = 0;        // 32 per-warp partials of a block sum
constexpr int kDslot = 32;     // 2 cluster-exchange slots of the partial log-likelihood
constexpr int kFlag = 38;      // decision word (as a double slot)
constexpr int kLogu = 40;      // log u of the next kLogBlock steps
constexpr int kLogBlock = 256;
constexpr int kNDouble = kLogu + kLogBlock;

template <typename R>
struct SeqMem {
    double *dbl;
    R *x, *g, *xt, *gt, *v, *mu, *slot, *part;  // vectors of kDMax; slot 2 x kDMax; part nthreads
    R *Xs, *ys, *cw, *Ps;                        // target data
};

template <typename R>
__device__ __forceinline__ SeqMem<R> carve(unsigned char *raw, const SeqCtx &c) {
    SeqMem<R> m;
    m.dbl = reinterpret_cast<double *>(raw);
    R *p = reinterpret_cast<R *>(raw + kNDouble * sizeof(double));
    m.x = p; p += kDMax;
    m.g = p; p += kDMax;
    m.xt = p; p += kDMax;
    m.gt = p; p += kDMax;
    m.v = p; p += kDMax;
    m.mu = p; p += kDMax;
    m.slot = p; p += 2 * kDMax;
    m.part = p; p += blockDim.x;
    m.Xs = m.ys = m.cw = m.Ps = nullptr;
    if (c.target == PMCMC_LOGREG) {
        m.Xs = p; p += (size_t)c.rows * c.Dp;
        m.ys = p; p += c.rows;
        m.cw = p; p += c.rows;
    } else {
        m.Ps = p; p += (size_t)c.D * c.Dp;
    }
    return m;
}

// A barrier over every thread of the chain's CTAs (the cluster when there is more than one).
__device__ __forceinline__ void chain_sync(int cs) {
    if (cs > 1)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

// Sum over the threads d < D of two doubles; every thread gets the results.
__device__ __forceinline__ void sum2(double a, double b, double *dbl, int D, double &ra, double &rb) {
    const int tid = threadIdx.x, w = tid >> 5;
    const int nw = (D + 31) >> 5;
    if (w < nw) {
        a = warp_sum(a);
        b = warp_sum(b);
        if ((tid & 31) == 0) {
            dbl[kRed + 2 * w] = a;
            dbl[kRed + 2 * w + 1] = b;
        }
    }
    __syncthreads();
    ra = 0.0;
    rb = 0.0;
    for (int i = 0; i < nw; i++) {
        ra += dbl[kRed + 2 * i];
        rb += dbl[kRed + 2 * i + 1];
    }
    __syncthreads();  // the partials may be overwritten afterwards
}

// Sum of a per-thread value over the CTA, returned to thread 0 only.  Double arithmetic is on
// GB300's narrow FP64 pipe (1/64 of the FP32 rate), so an FP32 value is summed as a compensated
// (hi, lo) pair (two-sum per step, exact up to the lo rounding) and only the per-warp pairs are
// added in FP64; a double value is summed in FP64.
__device__ __forceinline__ void two_sum(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}
__device__ __forceinline__ void warp_pair_sum(float &hi, float &lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        two_sum(hi, lo, h2);
        lo += l2;
    }
}
// exp(-|z|), 1 / (1 + e) and log(1 + e) for e in (0, 1]: hardware approximations in FP32 (as the
// parallel evaluate kernels use), library functions in FP64
__device__ __forceinline__ double exp_neg_abs(double z) { return exp(-fabs(z)); }
__device__ __forceinline__ float exp_neg_abs(float z) { return __expf(-fabsf(z)); }
__device__ __forceinline__ double recip1p(double e) { return 1.0 / (1.0 + e); }
__device__ __forceinline__ float recip1p(float e) { return __fdividef(1.0f, 1.0f + e); }
__device__ __forceinline__ double log1p_unit(double e) { return log1p(e); }
__device__ __forceinline__ float log1p_unit(float e) { return __logf(1.0f + e); }

template <typename R>
struct LLAcc {  // per-thread accumulator of log-likelihood terms
    double d = 0.0;
    __device__ __forceinline__ void add(R v) { d += (double)v; }
    __device__ __forceinline__ void to_warp_slot(double *slot) {
        d = warp_sum(d);
        if ((threadIdx.x & 31) == 0) *slot = d;
    }
};
template <>
struct LLAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v) { two_sum(hi, lo, v); }
    __device__ __forceinline__ void to_warp_slot(double *slot) {
        warp_pair_sum(hi, lo);
        if ((threadIdx.x & 31) == 0) *slot = (double)hi + (double)lo;
    }
};

// Logistic regression: likelihood gradient X^T (y - sigmoid(X v)) into out[0..D) (every CTA of
// the chain gets the full sum) and the log-likelihood sum_n y z - softplus(z) as the return value.
template <typename R>
__device__ double pass_logreg(const SeqCtx &c, const SeqMem<R> &m, const R *v, R *out, int buf) {
    const int tid = threadIdx.x, nt = blockDim.x, D = c.D;
    LLAcc<R> llp;
    for (int n = tid; n < c.rows; n += nt) {
        const R *xr = m.Xs + (size_t)n * c.Dp;
        R z = R(0);
        for (int d = 0; d < D; d++) z = fma(xr[d], v[d], z);
        const R e = exp_neg_abs(z);
        const R q = recip1p(e);
        const R p = z >= R(0) ? q : e * q;  // sigmoid(z)
        const R yv = m.ys[n];
        m.cw[n] = yv - p;
        llp.add(yv * z - (fmax(z, R(0)) + log1p_unit(e)));
    }
    llp.to_warp_slot(m.dbl + kRed + (tid >> 5));
    __syncthreads();
    for (int e = tid; e < c.K * D; e += nt) {
        const int k = e / D, d = e - k * D;
        R acc = R(0);
        for (int n = k; n < c.rows; n += c.K) acc = fma(m.cw[n], m.Xs[(size_t)n * c.Dp + d], acc);
        m.part[e] = acc;
    }
    __syncthreads();
    R *slot = m.slot + buf * kDMax;
    for (int d = tid; d < D; d += nt) {
        R s = R(0);
        for (int k = 0; k < c.K; k++) s += m.part[k * D + d];
        slot[d] = s;
    }
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (nt >> 5); w++) s += m.dbl[kRed + w];
        m.dbl[kDslot + buf] = s;
    }
    chain_sync(c.cs);
    double ll = 0.0;
    if (c.cs > 1) {
        cg::cluster_group cl = cg::this_cluster();
        for (int d = tid; d < D; d += nt) {
            R s = R(0);
            for (int r = 0; r < c.cs; r++) s += cl.map_shared_rank(slot, r)[d];
            out[d] = s;
        }
        for (int r = 0; r < c.cs; r++) ll += cl.map_shared_rank(m.dbl + kDslot + buf, r)[0];
    } else {
        for (int d = tid; d < D; d += nt) out[d] = slot[d];
        ll = m.dbl[kDslot + buf];
    }
    __syncthreads();
    return ll;
}

// Gaussian: gradient -P (v - mu) into out[0..D).
template <typename R>
__device__ __forceinline__ void pass_gauss(const SeqCtx &c, const SeqMem<R> &m, const R *v, R *out) {
    const int tid = threadIdx.x, D = c.D;
    if (tid < D) {
        const R *pr = m.Ps + (size_t)tid * c.Dp;
        R acc = R(0);
        for (int j = 0; j < D; j++) acc = fma(pr[j], v[j] - m.mu[j], acc);
        out[tid] = -acc;
    }
    __syncthreads();
}

template <typename R>
__device__ void run_chain(const SeqChain &ch, int cs, int rank, unsigned char *raw) {
    SeqCtx c;
    c.target = ch.target;
    c.sampler = ch.sampler;
    c.D = ch.D;
    c.N = ch.N;
    c.L = ch.L;
    c.T = ch.T;
    c.Dp = ch.D | 1;
    c.cs = cs;
    c.rank = rank;
    const int per = (ch.N + cs - 1) / cs;
    c.row0 = min(ch.N, rank * per);
    c.rows = max(0, min(ch.N, c.row0 + per) - c.row0);
    c.K = max(1, (int)blockDim.x / max(1, ch.D));
    const SeqMem<R> m = carve<R>(raw, c);
    const int tid = threadIdx.x, nt = blockDim.x, D = c.D;
    const bool lr = c.target == PMCMC_LOGREG;
    const R eps = (R)ch.eps;
    const R inv_sp2 = lr ? (R)(1.0 / (ch.sigma_p * ch.sigma_p)) : R(0);
    const double inv2sp = lr ? 0.5 / (ch.sigma_p * ch.sigma_p) : 0.0;

    // stage the target
    if (lr) {
        const R *X = static_cast<const R *>(ch.X), *y = static_cast<const R *>(ch.y);
        for (int e = tid; e < c.rows * D; e += nt) {
            const int n = e / D, d = e - n * D;
            m.Xs[(size_t)n * c.Dp + d] = X[(size_t)(c.row0 + n) * D + d];
        }
        for (int n = tid; n < c.rows; n += nt) m.ys[n] = y[c.row0 + n];
    } else {
        const R *P = static_cast<const R *>(ch.P), *mu = static_cast<const R *>(ch.mu);
        for (int e = tid; e < D * D; e += nt) {
            const int i = e / D, j = e - i * D;
            m.Ps[(size_t)i * c.Dp + j] = P[e];
        }
        for (int d = tid; d < D; d += nt) m.mu[d] = mu[d];
    }
    for (int d = tid; d < D; d += nt) m.x[d] = static_cast<const R *>(ch.s0)[d];
    chain_sync(cs);  // remote CTAs' shared memory is in use from here on

    // gradient and log-density at x (carried from step to step)
    int buf = 0;
    double lpx;  // log p(x) up to a constant
    {
        double ll = 0.0;
        if (lr) {
            ll = pass_logreg<R>(c, m, m.x, m.g, buf);
            buf ^= 1;
        } else {
            pass_gauss<R>(c, m, m.x, m.g);
        }
        double a = 0.0, b = 0.0;
        if (tid < D) {
            if (lr) {
                a = -(double)m.x[tid] * (double)m.x[tid] * inv2sp;
                m.g[tid] -= m.x[tid] * inv_sp2;
            } else {
                a = 0.5 * (double)(m.x[tid] - m.mu[tid]) * (double)m.g[tid];
            }
        }
        double ra, rb;
        sum2(a, b, m.dbl, D, ra, rb);
        lpx = ll + ra;
    }

    const R *xin = static_cast<const R *>(ch.xi);
    R *sout = static_cast<R *>(ch.s_out);
    const bool writer = rank == 0;
    R xi_cur = tid < D ? xin[tid] : R(0);
    const R sq = sqrt(R(2) * eps);

    for (int t = 0; t < c.T; t++) {
        // log u of the next kLogBlock steps, one per thread, off the per-step critical path
        if ((t % kLogBlock) == 0) {
            for (int i = tid; i < kLogBlock; i += nt)
                m.dbl[kLogu + i] = t + i < c.T ? log(ch.u[t + i]) : 0.0;
            __syncthreads();
        }
        // prefetch the next step's noise
        R xi_nxt = R(0);
        if (t + 1 < c.T && tid < D) xi_nxt = xin[(size_t)(t + 1) * D + tid];
        double gap = 0.0;  // log alpha-type quantity compared with log u: ell (MALA) or H0 - HL (HMC)
        double lpt = 0.0;  // log p at the proposal
        if (c.sampler == PMCMC_MALA) {
            if (tid < D) m.xt[tid] = m.x[tid] + eps * m.g[tid] + sq * xi_cur;
            __syncthreads();
            double ll = 0.0;
            if (lr) {
                ll = pass_logreg<R>(c, m, m.xt, m.gt, buf);
                buf ^= 1;
            } else {
                pass_gauss<R>(c, m, m.xt, m.gt);
            }
            double a = 0.0, b = 0.0;
            if (tid < D) {
                const R xt = m.xt[tid], x = m.x[tid];
                double lpd;
                if (lr) {
                    lpd = -(double)xt * (double)xt * inv2sp;
                    m.gt[tid] -= xt * inv_sp2;
                } else {
                    lpd = 0.5 * (double)(xt - m.mu[tid]) * (double)m.gt[tid];
                }
                const double e = (double)x - (double)xt - (double)eps * (double)m.gt[tid];
                a = lpd;
                b = -e * e / (4.0 * (double)eps) + 0.5 * (double)xi_cur * (double)xi_cur;
            }
            double ra, rb;
            sum2(a, b, m.dbl, D, ra, rb);
            lpt = ll + ra;
            gap = lpt - lpx + rb;  // ell
        } else {
            // HMC: v0 = xi, half step, L leapfrog steps, undo the last half step (Algorithm 2)
            if (tid < D) {
                m.xt[tid] = m.x[tid];
                m.v[tid] = xi_cur + R(0.5) * eps * m.g[tid];
            }
            double ll = 0.0;
            const R *glast = m.g;
            for (int k = 0; k < c.L; k++) {
                if (tid < D) m.xt[tid] += eps * m.v[tid];
                __syncthreads();
                if (lr) {
                    ll = pass_logreg<R>(c, m, m.xt, m.gt, buf);
                    buf ^= 1;
                    if (tid < D) m.gt[tid] -= m.xt[tid] * inv_sp2;
                } else {
                    pass_gauss<R>(c, m, m.xt, m.gt);
                }
                if (tid < D) m.v[tid] += eps * m.gt[tid];
                glast = m.gt;
            }
            double a = 0.0, b = 0.0;
            if (tid < D) {
                m.v[tid] -= R(0.5) * eps * glast[tid];
                const R xt = m.xt[tid];
                a = lr ? -(double)xt * (double)xt * inv2sp
                       : 0.5 * (double)(xt - m.mu[tid]) * (double)glast[tid];
                b = 0.5 * (double)xi_cur * (double)xi_cur - 0.5 * (double)m.v[tid] * (double)m.v[tid];
            }
            double ra, rb;
            sum2(a, b, m.dbl, D, ra, rb);
            lpt = (c.L > 0 ? ll : 0.0) + ra;
            if (c.L == 0) lpt = lpx;
            // H0 - HL = (|xi|^2/2 - lp(x0)) - (|vL|^2/2 - lp(xL))
            gap = rb - lpx + lpt;
        }
        if (tid == 0) {
            const double la = (gap < 0.0 || isnan(gap)) ? gap : 0.0;
            m.dbl[kFlag] = (la - m.dbl[kLogu + t % kLogBlock] > 0.0) ? 1.0 : 0.0;
        }
        __syncthreads();
        const bool acc = m.dbl[kFlag] != 0.0;
        if (acc) {
            if (tid < D) {
                m.x[tid] = m.xt[tid];
                m.g[tid] = (c.sampler == PMCMC_HMC && c.L == 0) ? m.g[tid] : m.gt[tid];
            }
            lpx = lpt;
        }
        if (writer) {
            if (tid < D) sout[(size_t)t * D + tid] = acc ? m.xt[tid] : m.x[tid];
            if (tid == 0 && ch.acc_out) ch.acc_out[t] = acc ? 1 : 0;
        }
        xi_cur = xi_nxt;
        __syncthreads();  // x and g settled before the next proposal reads them
    }
    chain_sync(cs);  // no CTA leaves while another may still read its shared memory
}

// One chain per cluster of cs CTAs (cluster launch, gridDim = cs).
template <typename R>
__global__ void __launch_bounds__(kSeqThreads, 1) seq_chain_kernel(SeqChain one, int cs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rank = cs > 1 ? (int)cg::this_cluster().block_rank() : 0;
    run_chain<R>(one, cs, rank, smem_raw);
}

// One chain per CTA, many chains per launch (several CTAs resident per SM).
template <typename R>
__global__ void __launch_bounds__(kSeqThreadsBatched, 3) seq_chains_kernel(const SeqChain *many) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    run_chain<R>(many[blockIdx.x], 1, 0, smem_raw);
}

}  // namespace

size_t seq_smem_bytes(const SeqChain &ch, int cs, int threads, bool f64) {
    const size_t rb = f64 ? 8 : 4;
    const int Dp = ch.D | 1;
    size_t r = (size_t)kNDouble * 8 + rb * ((size_t)8 * kDMax + threads);
    if (ch.target == PMCMC_LOGREG) {
        const int rows = (ch.N + cs - 1) / cs;
        r += rb * ((size_t)rows * Dp + 2 * (size_t)rows);
    } else {
        r += rb * (size_t)ch.D * Dp;
    }
    return r;
}

SeqChain seq_chain_from(const EvalArgs &A) {
    SeqChain ch;
    ch.target = A.target;
    ch.sampler = A.sampler;
    ch.D = A.D;
    ch.N = A.N;
    ch.L = A.L;
    ch.T = A.T;
    ch.eps = A.eps;
    ch.sigma_p = A.sigma_p;
    ch.X = A.X;
    ch.y = A.y;
    ch.mu = A.mu;
    ch.P = A.P;
    ch.s0 = A.s0;
    ch.xi = A.xi;
    ch.u = A.u;
    ch.s_out = A.f_out;
    ch.acc_out = A.acc_out;
    return ch;
}

bool seq_fast_supported(const SeqChain &ch) {
    if (ch.sampler != PMCMC_MALA && ch.sampler != PMCMC_HMC) return false;
    if (ch.target != PMCMC_LOGREG && ch.target != PMCMC_GAUSSIAN) return false;
    return ch.D >= 1 && ch.D <= kDMax && ch.T >= 1;
}

// Cluster size of a single chain: the smallest power of two whose row share fits the shared
// memory budget of one SM, at least 1 and at most 16 (PMCMC_SEQ_CLUSTER overrides, for
// measurements).  Returns 0 when even 16 CTAs cannot hold the design.
int seq_cluster_size(const SeqChain &ch, bool f64) {
    const char *e = getenv("PMCMC_SEQ_CLUSTER");
    if (e && atoi(e) >= 1 && atoi(e) <= 16) {
        const int v = atoi(e);
        return seq_smem_bytes(ch, v, kSeqThreads, f64) <= kSeqSmemBudget ? v : 0;
    }
    for (int cs = 1; cs <= 16; cs *= 2)
        if (seq_smem_bytes(ch, cs, kSeqThreads, f64) <= kSeqSmemBudget) return cs;
    return 0;
}

cudaError_t launch_seq_chain(const SeqChain &ch, bool f64, cudaStream_t st) {
    const int cs = seq_cluster_size(ch, f64);
    if (cs == 0) return cudaErrorInvalidValue;
    const size_t sm = seq_smem_bytes(ch, cs, kSeqThreads, f64);
    auto k = f64 ? seq_chain_kernel<double> : seq_chain_kernel<float>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kSeqThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, ch, cs);
}

cudaError_t launch_seq_chains(const SeqChain *dev_chains, int B, size_t smem, bool f64,
                              cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    if (smem > kSeqSmemBudget) return cudaErrorInvalidValue;
    auto k = f64 ? seq_chains_kernel<double> : seq_chains_kernel<float>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<B, kSeqThreadsBatched, smem, st>>>(dev_chains);
    return cudaGetLastError();
}

}  // namespace pm
