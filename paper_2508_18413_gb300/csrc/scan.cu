// Parallel affine scans (the linear solve of each Newton iteration, Section 2 and Eqs. 3-4):
//   delta_t = A_t delta_{t-1} + b_t,  delta_{-1} = 0,   s_t <- s_t + delta_t.
// Composing affine maps is associative: (A2, b2) o (A1, b1) = (A2 A1, A2 b1 + b2).
//
// Both kernels are single-pass with a decoupled look-back: each CTA takes a tile (ticketed, so
// a CTA only ever waits on tiles that were dispatched before it), publishes its tile aggregate,
// looks back for the nearest predecessor whose inclusive result is published, evaluates the
// carry forward through the intervening aggregates (matrix-vector products only), publishes its
// own inclusive result and applies the carry.  Every wait is bounded: when a wait runs out the
// CTA records a timeout in the control block and continues, so no launch can hang.
//
// A non-finite updated element is reset (to s_reset, or 0): the fixed point is finite, and an
// iterate poisoned by an overflow would otherwise stop the Newton iteration from progressing.
#include "common.cuh"
#include "internal.h"

namespace pm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kFlagAgg = 1, kFlagIncl = 2;

__device__ __forceinline__ int smem_idx(int e) { return e + (e >> 5); }  // pad 1 word / 32

__device__ __forceinline__ unsigned int take_tile(ScanCtl *ctl, unsigned int *s_tile,
                                                  unsigned int *s_epoch) {
    if (threadIdx.x == 0) {
        *s_tile = atomicAdd(&ctl->ticket, 1u);
        *s_epoch = *(volatile unsigned int *)&ctl->epoch;
    }
    __syncthreads();
    return *s_tile;
}

__device__ __forceinline__ void finish_tile(ScanCtl *ctl, unsigned int ntiles) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int d = atomicAdd(&ctl->done, 1u);
        if (d == ntiles - 1) {  // last CTA: reset for the next launch
            ctl->ticket = 0;
            ctl->done = 0;
            ctl->epoch = ctl->epoch + 1u;
            __threadfence();
        }
    }
}

// Wait (bounded) until tile j's flag carries this epoch; returns the state (0 on timeout).
__device__ __forceinline__ unsigned int wait_flag(const unsigned int *flags, int j,
                                                  unsigned int epoch, unsigned int limit,
                                                  ScanCtl *ctl) {
    Spin spin(limit);
    for (;;) {
        unsigned int f = ld_acquire(flags + j);
        if ((f >> 2) == (epoch & 0x3fffffffu) && (f & 3u)) return f & 3u;
        if (!spin.again()) {
            atomicExch(&ctl->timeout, 1u);
            return 0;
        }
    }
}

__device__ __forceinline__ unsigned int make_flag(unsigned int epoch, unsigned int state) {
    return ((epoch & 0x3fffffffu) << 2) | state;
}

}  // namespace

// ==========================================================================================
// Diagonal scan: D independent channels, elementwise maps.  Tile = TT timesteps x D channels,
// staged through shared memory; thread (j, d) scans segment j of channel d.
// ==========================================================================================
template <typename R, typename S>
__global__ void __launch_bounds__(kScanThreads)
scan_diag_kernel(int T, int D, int TT, const S *__restrict__ a, const S *__restrict__ b,
                 R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                 R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl, EvalStats *stats,
                 const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    extern __shared__ unsigned char smem_raw[];
    __shared__ unsigned int s_tile, s_epoch;
    const unsigned int ntiles = (unsigned int)ceil_div(T, TT);
    const int tile = (int)take_tile(ctl, &s_tile, &s_epoch);
    const unsigned int epoch = s_epoch;

    const int E = TT * D;
    const int Ep = smem_idx(E) + 1;
    R *sa = reinterpret_cast<R *>(smem_raw);
    R *sb = sa + Ep;
    R *ss = sb + Ep;
    R *segA = ss + Ep;             // NS * D
    R *segB = segA + kScanThreads; // NS * D
    R *carry = segB + kScanThreads;  // D

    const int t0 = tile * TT;
    const int TTv = min(TT, T - t0);
    const int Ev = TTv * D;
    const size_t base = (size_t)t0 * D;
    const int tid = threadIdx.x;

    for (int e = tid; e < Ev; e += kScanThreads) {
        const int k = smem_idx(e);
        sa[k] = load_as<S, R>(a + base + e);
        sb[k] = load_as<S, R>(b + base + e);
        ss[k] = s[base + e];
    }
    __syncthreads();

    const int NS = max(1, kScanThreads / D);
    const int klen = ceil_div(TT, NS);
    const int j = tid / D, d = tid - (tid / D) * D;
    const bool active = j < NS;
    const int i0 = j * klen, i1 = min(i0 + klen, TTv);

    // Phase A: segment aggregates
    R A = R(1), B = R(0);
    if (active) {
        for (int i = i0; i < i1; i++) {
            const int k = smem_idx(i * D + d);
            const R ai = sa[k];
            B = ai * B + sb[k];
            A = ai * A;
        }
    }
    // Phase B: inclusive scan over segments of each channel (Hillis-Steele)
    for (int off = 1; off < NS; off <<= 1) {
        if (active) {
            segA[tid] = A;
            segB[tid] = B;
        }
        __syncthreads();
        if (active && j >= off) {
            const R pa = segA[tid - off * D], pb = segB[tid - off * D];
            B = A * pb + B;
            A = A * pa;
        }
        __syncthreads();
    }
    if (active) {
        segA[tid] = A;
        segB[tid] = B;
    }
    __syncthreads();

    // Phase C: publish the tile aggregate, look back, publish the inclusive result.
    const int last = (NS - 1) * D;
    if (tid < D) {
        const R TA = segA[last + tid], TB = segB[last + tid];
        if (tile == 0) {
            gincl[(size_t)tile * D + tid] = TB;
        } else {
            gagg[((size_t)tile * 2) * D + tid] = TA;
            gagg[((size_t)tile * 2 + 1) * D + tid] = TB;
        }
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) st_release(flags + tile, make_flag(epoch, tile == 0 ? kFlagIncl : kFlagAgg));
    if (tile > 0 && tid < D) {
        // walk back to the nearest inclusive predecessor
        int jj = tile - 1;
        for (; jj >= 0; jj--) {
            unsigned int st = wait_flag(flags, jj, epoch, spin_limit, ctl);
            if (st == kFlagIncl || st == 0) break;
        }
        R c = R(0);
        if (jj >= 0) {
            unsigned int st = ld_acquire(flags + jj);
            if ((st & 3u) == kFlagIncl && (st >> 2) == (epoch & 0x3fffffffu))
                c = gincl[(size_t)jj * D + tid];
        }
        for (int m = max(jj + 1, 0); m < tile; m++) {  // carry forward through aggregates
            const R ma = gagg[((size_t)m * 2) * D + tid], mb = gagg[((size_t)m * 2 + 1) * D + tid];
            c = ma * c + mb;
        }
        carry[tid] = c;
        const R TA = segA[last + tid], TB = segB[last + tid];
        gincl[(size_t)tile * D + tid] = TA * c + TB;
        __threadfence();
    } else if (tile == 0 && tid < D) {
        carry[tid] = R(0);
    }
    __syncthreads();
    if (tile > 0 && tid == 0) st_release(flags + tile, make_flag(epoch, kFlagIncl));

    // Phase D: apply the carry and update the state.
    R dmax = R(0);
    unsigned int resets = 0;
    if (active && i0 < i1) {
        R delta = carry[d];
        if (j > 0) {
            const R pa = segA[tid - D], pb = segB[tid - D];
            delta = pa * delta + pb;
        }
        for (int i = i0; i < i1; i++) {
            const int k = smem_idx(i * D + d);
            delta = sa[k] * delta + sb[k];
            R sn = ss[k] + delta;
            if (!finite(sn)) {
                sn = s_reset ? s_reset[d] : R(0);
                resets++;
            } else {
                dmax = max(dmax, fabs(delta));
            }
            ss[k] = sn;
        }
    }
    __syncthreads();
    for (int e = tid; e < Ev; e += kScanThreads) s[base + e] = ss[smem_idx(e)];

    if (stats) {
        double dm = warp_max((double)dmax);
        unsigned int rs = warp_sum(resets);
        if ((tid & 31) == 0) {
            if (dm > 0) atomic_max_d(&stats->dmax, dm);
            if (rs) atomicAdd(&stats->resets, (unsigned long long)rs);
        }
    }
    finish_tile(ctl, ntiles);
}

int diag_scan_tile(int T, int D, int elem_bytes) {
    // enough tiles to fill the GPU twice over, at most ~4096 elements (FP32) per tile
    const int max_elems = elem_bytes >= 8 ? 2048 : 4096;
    int tt_max = std::max(8, (max_elems / std::max(D, 1)) / 8 * 8);
    int tt = ceil_div(T, 2 * 152);
    tt = (tt + 7) / 8 * 8;
    tt = std::max(8, std::min(tt, tt_max));
    return tt;
}

static size_t diag_smem(int TT, int D, int rbytes) {
    int E = TT * D;
    int Ep = E + (E >> 5) + 1;
    return (size_t)rbytes * (3 * (size_t)Ep + 2 * kScanThreads + D + 4);
}

template <typename R, typename S>
static cudaError_t run_scan_diag(int T, int D, int TT, const void *a, const void *b, void *s,
                                 const void *s_reset, const ScanWork &w, EvalStats *stats,
                                 const int *skip, unsigned int spin, cudaStream_t st) {
    const int ntiles = ceil_div(T, TT);
    size_t sm = diag_smem(TT, D, sizeof(R));
    auto k = scan_diag_kernel<R, S>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k<<<ntiles, kScanThreads, sm, st>>>(T, D, TT, (const S *)a, (const S *)b, (R *)s,
                                        (const R *)s_reset, w.flags, (R *)w.agg, (R *)w.incl,
                                        w.ctl, stats, skip, spin);
    return cudaGetLastError();
}

cudaError_t launch_scan_diag(bool f64, int storage, int T, int D, int tile_t, const void *a,
                             const void *b, void *s, const void *s_reset, const ScanWork &w,
                             EvalStats *stats, const int *skip, unsigned int spin_limit,
                             cudaStream_t st) {
    if (ceil_div(T, tile_t) > w.max_tiles) return cudaErrorInvalidValue;
    if (f64) return run_scan_diag<double, double>(T, D, tile_t, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    if (storage == 1)
        return run_scan_diag<float, __nv_bfloat16>(T, D, tile_t, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    return run_scan_diag<float, float>(T, D, tile_t, a, b, s, s_reset, w, stats, skip, spin_limit, st);
}

// ==========================================================================================
// Dense scan (DEER, Eq. 3), D <= 32: one CTA per chunk of C timesteps.
//   Phase A: chunk aggregate (Phi, beta) = composition of its (J_t, b_t), sequential matmuls.
//   Phase C: look-back; the carry is evaluated forward with matrix-vector products.
//   Phase D: re-run the recursion from the carry (matrix-vector products), update s.
// ==========================================================================================
template <typename R, int DM>
__global__ void __launch_bounds__(kScanThreads)
scan_dense_kernel(int T, int D, int C, const R *__restrict__ a, const R *__restrict__ b,
                  R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                  R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl, EvalStats *stats,
                  const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    __shared__ R Phi[2][DM * DM];
    __shared__ R Jt[DM * DM];
    __shared__ R beta[2][DM];
    __shared__ R vec[2][DM];
    __shared__ unsigned int s_tile, s_epoch;
    const unsigned int ntiles = (unsigned int)ceil_div(T, C);
    const int tile = (int)take_tile(ctl, &s_tile, &s_epoch);
    const unsigned int epoch = s_epoch;
    const int tid = threadIdx.x;
    const int DD = D * D;
    const int t0 = tile * C;
    const int Cv = min(C, T - t0);
    const size_t AGG = (size_t)DD + D;

    // Phase A
    for (int e = tid; e < DD; e += kScanThreads) Phi[0][e] = (e / D == e % D) ? R(1) : R(0);
    if (tid < D) beta[0][tid] = R(0);
    __syncthreads();
    int cur = 0;
    for (int i = 0; i < Cv; i++) {
        const R *Ji = a + (size_t)(t0 + i) * DD;
        for (int e = tid; e < DD; e += kScanThreads) Jt[e] = Ji[e];
        __syncthreads();
        for (int e = tid; e < DD; e += kScanThreads) {
            const int r = e / D, c = e - r * D;
            R acc = R(0);
            for (int k = 0; k < D; k++) acc += Jt[r * D + k] * Phi[cur][k * D + c];
            Phi[cur ^ 1][e] = acc;
        }
        if (tid < D) {
            R acc = b[(size_t)(t0 + i) * D + tid];
            for (int k = 0; k < D; k++) acc += Jt[tid * D + k] * beta[cur][k];
            beta[cur ^ 1][tid] = acc;
        }
        __syncthreads();
        cur ^= 1;
    }

    // Phase C
    if (tile == 0) {
        if (tid < D) gincl[tid] = beta[cur][tid];
        __threadfence();
    } else {
        for (int e = tid; e < DD; e += kScanThreads) gagg[(size_t)tile * AGG + e] = Phi[cur][e];
        if (tid < D) gagg[(size_t)tile * AGG + DD + tid] = beta[cur][tid];
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) st_release(flags + tile, make_flag(epoch, tile == 0 ? kFlagIncl : kFlagAgg));
    __shared__ int s_jj;
    if (tile > 0) {
        if (tid == 0) {
            int jj = tile - 1;
            for (; jj >= 0; jj--) {
                unsigned int st = wait_flag(flags, jj, epoch, spin_limit, ctl);
                if (st == kFlagIncl || st == 0) break;
            }
            if (jj >= 0) {
                unsigned int st = ld_acquire(flags + jj);
                if (!((st & 3u) == kFlagIncl && (st >> 2) == (epoch & 0x3fffffffu))) jj = -1;
            }
            s_jj = jj;
        }
        __syncthreads();
        const int jj = s_jj;
        int vc = 0;
        if (tid < D) vec[0][tid] = jj >= 0 ? gincl[(size_t)jj * D + tid] : R(0);
        __syncthreads();
        for (int m = max(jj + 1, 0); m < tile; m++) {
            const R *Am = gagg + (size_t)m * AGG;
            if (tid < D) {
                R acc = Am[DD + tid];
                for (int k = 0; k < D; k++) acc += Am[tid * D + k] * vec[vc][k];
                vec[vc ^ 1][tid] = acc;
            }
            __syncthreads();
            vc ^= 1;
        }
        // inclusive = Phi * carry + beta
        if (tid < D) {
            R acc = beta[cur][tid];
            for (int k = 0; k < D; k++) acc += Phi[cur][tid * D + k] * vec[vc][k];
            gincl[(size_t)tile * D + tid] = acc;
            vec[0][tid] = vec[vc][tid];  // carry
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(flags + tile, make_flag(epoch, kFlagIncl));
    } else {
        if (tid < D) vec[0][tid] = R(0);
        __syncthreads();
    }

    // Phase D: delta_t = J_t delta_{t-1} + b_t from the carry
    R dmax = R(0);
    unsigned int resets = 0;
    int vc = 0;
    for (int i = 0; i < Cv; i++) {
        const R *Ji = a + (size_t)(t0 + i) * DD;
        const size_t row = (size_t)(t0 + i) * D;
        if (tid < D) {
            R acc = b[row + tid];
            for (int k = 0; k < D; k++) acc += Ji[tid * D + k] * vec[vc][k];
            vec[vc ^ 1][tid] = acc;
            R sn = s[row + tid] + acc;
            if (!finite(sn)) {
                sn = s_reset ? s_reset[tid] : R(0);
                resets++;
            } else {
                dmax = max(dmax, fabs(acc));
            }
            s[row + tid] = sn;
        }
        __syncthreads();
        vc ^= 1;
    }
    if (stats && tid < 32) {
        double dm = warp_max((double)dmax);
        unsigned int rs = warp_sum(resets);
        if (tid == 0) {
            if (dm > 0) atomic_max_d(&stats->dmax, dm);
            if (rs) atomicAdd(&stats->resets, (unsigned long long)rs);
        }
    }
    finish_tile(ctl, ntiles);
}

int dense_scan_chunk(int T, int D) {
    int c = ceil_div(T, 2 * 152);
    return std::max(8, std::min(c, 64));
}

template <typename R, int DM>
static cudaError_t run_scan_dense(int T, int D, int C, const void *a, const void *b, void *s,
                                  const void *s_reset, const ScanWork &w, EvalStats *stats,
                                  const int *skip, unsigned int spin, cudaStream_t st) {
    scan_dense_kernel<R, DM><<<ceil_div(T, C), kScanThreads, 0, st>>>(
        T, D, C, (const R *)a, (const R *)b, (R *)s, (const R *)s_reset, w.flags, (R *)w.agg,
        (R *)w.incl, w.ctl, stats, skip, spin);
    return cudaGetLastError();
}

cudaError_t launch_scan_dense(bool f64, int T, int D, int chunk, const void *a, const void *b,
                              void *s, const void *s_reset, const ScanWork &w, EvalStats *stats,
                              const int *skip, unsigned int spin_limit, cudaStream_t st) {
    if (ceil_div(T, chunk) > w.max_tiles) return cudaErrorInvalidValue;
    if (D > 32) return cudaErrorInvalidValue;
#define PM_DENSE(R_, DM_) \
    return run_scan_dense<R_, DM_>(T, D, chunk, a, b, s, s_reset, w, stats, skip, spin_limit, st)
    if (f64) {
        if (D <= 4) PM_DENSE(double, 4);
        if (D <= 8) PM_DENSE(double, 8);
        if (D <= 16) PM_DENSE(double, 16);
        PM_DENSE(double, 32);
    } else {
        if (D <= 4) PM_DENSE(float, 4);
        if (D <= 8) PM_DENSE(float, 8);
        if (D <= 16) PM_DENSE(float, 16);
        PM_DENSE(float, 32);
    }
#undef PM_DENSE
}

}  // namespace pm
