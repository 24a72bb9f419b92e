// Decoupled look-back of the single-pass scans: per-tile flags tagged with a launch epoch, and
// the block-wide walk over windows of 64 predecessor tiles.  Shared by the scan kernels and the
// tensor-core evaluate kernel, which applies the Newton update in the same launch.
#pragma once

#include "common.cuh"

namespace pm {

constexpr int kFlagAgg = 1, kFlagIncl = 2;

// The barrier of the 256 threads that run a look-back: the whole CTA (the scan kernels) or a
// named barrier of a subset of its warps (kernels with other warp roles).
struct CtaBar {
    __device__ static void sync() { __syncthreads(); }
};
template <int kId>
struct NamedBar256 {
    __device__ static void sync() { asm volatile("bar.sync %0, 256;" ::"n"(kId) : "memory"); }
};

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

// Block-wide look-back over windows of 64 predecessors (all 256 threads, D <= 32 channels).
// Thread i examines predecessor p = i % 64 of the window for channel group g = i / 64
// (channels 8g .. 8g + 7), so one round of independent loads brings every channel of the whole
// window; only the 64 threads of group 0 poll the flags.  The nearest predecessor with a
// published inclusive value (or tile -1, or a timed-out wait) ends the walk; the aggregates in
// between are composed per channel by a shuffle tree in each warp (lower lane = nearer, later
// map) and then across the two warps of the group.  Returns the carry of channel d in shared
// carry_out[d].
template <typename R, class Bar = CtaBar>
__device__ void lookback_block64(const unsigned int *flags, const R *gagg, const R *gincl, int tile,
                                 int D, unsigned int epoch, unsigned int spin_limit, ScanCtl *ctl,
                                 R *carry_out) {
    __shared__ int s_k;
    __shared__ unsigned int s_st[64];
    __shared__ R s_wa[2][32], s_wb[2][32], s_iv[32], s_MA[32], s_MB[32];
    const int tid = threadIdx.x, lane = tid & 31;
    const int pj = tid & 63, g = tid >> 6, half = pj >> 5;
    if (tid < 32) {
        s_MA[tid] = R(1);
        s_MB[tid] = R(0);
    }
    int jend = tile - 1;
    for (;;) {
        if (tid == 0) s_k = 64;
        Bar::sync();
        const int j = jend - pj;
        if (g == 0) {
            unsigned int st = kFlagIncl;
            if (j >= 0) st = wait_flag(flags, j, epoch, spin_limit, ctl);
            s_st[pj] = st;
            if (j < 0 || st != kFlagAgg) atomicMin(&s_k, pj);
        }
        Bar::sync();
        const int k = s_k;
        const unsigned int st = s_st[pj];
        if (k < 64 && pj == k) {
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const int d = 8 * g + c;
                if (d < D) s_iv[d] = (j >= 0 && st == kFlagIncl) ? gincl[(size_t)j * D + d] : R(0);
            }
        }
        R ga[8], gb[8];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int d = 8 * g + c;
            const bool on = pj < k && d < D;
            ga[c] = on ? gagg[((size_t)j * 2) * D + d] : R(1);
            gb[c] = on ? gagg[((size_t)j * 2 + 1) * D + d] : R(0);
        }
#pragma unroll
        for (int c = 0; c < 8; c++) {
            R a = ga[c], b = gb[c];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const R oa = __shfl_down_sync(0xffffffffu, a, off);
                const R ob = __shfl_down_sync(0xffffffffu, b, off);
                if (lane + off < 32) {
                    b = a * ob + b;
                    a = a * oa;
                }
            }
            const int d = 8 * g + c;
            if (lane == 0 && d < D) {
                s_wa[half][d] = a;
                s_wb[half][d] = b;
            }
        }
        Bar::sync();
        if (tid < D) {
            // window map W = half 0 o half 1 (half 0 holds the nearer predecessors)
            const R Wb = s_wa[0][tid] * s_wb[1][tid] + s_wb[0][tid];
            const R Wa = s_wa[0][tid] * s_wa[1][tid];
            const R MA = s_MA[tid], MB = s_MB[tid];  // M <- M o W
            s_MB[tid] = MA * Wb + MB;
            s_MA[tid] = MA * Wa;
            if (k < 64) carry_out[tid] = s_MA[tid] * s_iv[tid] + s_MB[tid];
        }
        Bar::sync();
        if (k < 64) break;
        jend -= 64;
    }
}

// Shared-memory values per aggregate staged by lookback_dense: D rows of D + 1 (padded) and b.
__host__ __device__ constexpr int dense_stage_stride(int D) { return D * (D + 1) + D; }

// Dense look-back (D <= 32; tile aggregates are affine maps (A, b), A row-major, D * D + D
// values per tile in gagg; inclusive values D per tile in gincl).  Warp 0 finds the nearest
// predecessor with a published inclusive value, 32 flags per round (a ballot picks the nearest
// lane that saw an inclusive flag or ran past tile 0).  The aggregates of the tiles in between
// are then staged into shared memory `stage` (nb of them at a time, dense_stage_stride(D)
// values each; all threads load, each a whole row, rows padded to D + 1 so that lane r reading
// row r is free of bank conflicts) and warp 0 applies them in order as matrix-vector products,
// the vector held one component per lane.  A timed-out wait (recorded in ctl) leaves a zero
// carry.  The carry of component d ends in carry_out[d].  Called by all threads of the block
// (NT of them, Bar their barrier).
template <typename R, int NT, class Bar = CtaBar>
__device__ void lookback_dense(const unsigned int *flags, const R *gagg, const R *gincl, int tile,
                               int D, unsigned int epoch, unsigned int spin_limit, ScanCtl *ctl,
                               R *stage, int nb, R *carry_out) {
    __shared__ int s_jj;
    const int tid = threadIdx.x, lane = tid & 31;
    const int DD = D * D, SQ = dense_stage_stride(D);
    const size_t AGG = (size_t)DD + D;
    if (tid < 32) {
        int jend = tile - 1, jj = -1;
        bool timed_out = false;
        for (;;) {
            const int j = jend - lane;
            unsigned int st = kFlagIncl;  // j < 0: the walk ran past tile 0
            if (j >= 0) st = wait_flag(flags, j, epoch, spin_limit, ctl);
            const unsigned int stop = __ballot_sync(0xffffffffu, j < 0 || st != kFlagAgg);
            if (stop) {
                const int l = __ffs(stop) - 1;
                const unsigned int stl = __shfl_sync(0xffffffffu, st, l);
                jj = jend - l;
                timed_out = jj >= 0 && stl != kFlagIncl;
                break;
            }
            jend -= 32;
        }
        if (lane == 0) s_jj = timed_out ? -2 : jj;
    }
    Bar::sync();
    const int jj = s_jj;
    R v = R(0);  // warp 0: component `lane` of the running vector
    if (tid < 32 && jj >= 0 && lane < D) v = __ldcg(gincl + (size_t)jj * D + lane);
    for (int m0 = (jj == -2 ? tile : jj + 1); m0 < tile; m0 += nb) {
        const int cnt = min(nb, tile - m0);
        // stage rows: (aggregate q, row r), r == D is b
        for (int idx = tid; idx < cnt * (D + 1); idx += NT) {
            const int q = idx / (D + 1), r = idx - q * (D + 1);
            const R *src = gagg + (size_t)(m0 + q) * AGG + (size_t)r * D;
            R *dst = stage + (size_t)q * SQ + r * (D + 1);
            R tmp[32];
#pragma unroll
            for (int c = 0; c < 32; c++) tmp[c] = c < D ? __ldcg(src + c) : R(0);
#pragma unroll
            for (int c = 0; c < 32; c++)
                if (c < D) dst[c] = tmp[c];
        }
        Bar::sync();
        if (tid < 32) {
            for (int q = 0; q < cnt; q++) {
                const R *Aq = stage + (size_t)q * SQ;
                R acc0 = lane < D ? Aq[D * (D + 1) + lane] : R(0), acc1 = R(0);
#pragma unroll
                for (int k = 0; k < 32; k += 2) {
                    const R v0 = __shfl_sync(0xffffffffu, v, k), v1 = __shfl_sync(0xffffffffu, v, k + 1);
                    if (k < D && lane < D) acc0 = fma(Aq[lane * (D + 1) + k], v0, acc0);
                    if (k + 1 < D && lane < D) acc1 = fma(Aq[lane * (D + 1) + k + 1], v1, acc1);
                }
                v = lane < D ? acc0 + acc1 : R(0);
            }
        }
        Bar::sync();
    }
    if (tid < D) carry_out[tid] = v;
    Bar::sync();
}

}  // namespace pm
