// Decoupled look-back of the single-pass scans: per-tile flags tagged with a launch epoch, and
// the block-wide walk over windows of 64 predecessor tiles.  Shared by the scan kernels and the
// tensor-core evaluate kernel, which applies the Newton update in the same launch.
#pragma once

#include "common.cuh"
#include "tc.cuh"

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

// Stride of a tile's aggregate (A row-major, then b: D * D + D values) in the dense look-back's
// aggregate array, rounded up to a multiple of 4 values so that every aggregate starts on a
// 16-byte boundary and a run of them is one bulk copy.
__host__ __device__ constexpr int dense_agg_stride(int D) { return (D * D + D + 3) & ~3; }

// Dense look-back (D <= 32; tile aggregates are affine maps (A, b) stored at dense_agg_stride(D)
// values per tile in gagg; inclusive values D per tile in gincl), run by warp 0 of the block.
// The warp finds the nearest predecessor with a published inclusive value, 32 flags per round
// (a ballot picks the nearest lane that saw an inclusive flag or ran past tile 0).  The
// aggregates of the tiles in between are a contiguous run of gagg: lane 0 stages it into shared
// memory by bulk copies (cp.async.bulk, completing on the two mbarriers at bars, bars + 8) in
// batches of up to nb aggregates, double-buffered so that the next batch is in flight while the
// warp applies the current one as matrix-vector products (the vector held one component per
// lane).  Lane r reads row r of A starting at column r and wrapping around, so at D = 32 the 32
// lanes read 32 different banks; the rotated columns are computed once per call (with D known
// only at run time, recomputing them per step made each product ~2.7x slower, measured).  A wait that runs out (recorded in ctl) leaves a zero carry;
// copies in flight are drained before return.  The carry of component d ends in carry_out[d].
// Called by all threads of the block (Bar their barrier); stage holds 2 nb aggregates.
template <typename R, class Bar = CtaBar>
__device__ void lookback_dense(const unsigned int *flags, const R *gagg, const R *gincl, int tile,
                               int D, unsigned int epoch, unsigned int spin_limit, ScanCtl *ctl,
                               R *stage, int nb, uint32_t bars, R *carry_out) {
    static_assert(sizeof(R) == 4, "four-byte values");
    const int tid = threadIdx.x, lane = tid & 31;
    const int DD = D * D, AS = dense_agg_stride(D);
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
        R v = R(0);  // component `lane` of the running vector
        if (!timed_out && jj >= 0 && lane < D) v = __ldcg(gincl + (size_t)jj * D + lane);
        const int m0 = timed_out ? tile : jj + 1;
        const uint32_t sbase = tc::smem_u32(stage);
        // the flags were acquired by the warp's lanes: order them before lane 0's copies, and
        // the aggregates they publish (generic stores) before the copies' reads (async proxy)
        // (one fence covers every copy: all the aggregates they read were published before the
        // flags the walk observed)
        __syncwarp();
        if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        auto issue = [&](int buf, int m) {  // lane 0: aggregates m .. m + cnt - 1 into buffer buf
            const int cnt = min(nb, tile - m);
            const uint32_t bytes = (uint32_t)(cnt * AS * (int)sizeof(R));
            tc::mbar_arrive_expect_tx(bars + 8u * (uint32_t)buf, bytes);
            tc::bulk_g2s(sbase + (uint32_t)(buf * nb * AS * (int)sizeof(R)), gagg + (size_t)m * AS, bytes,
                         bars + 8u * (uint32_t)buf);
        };
        // lane r reads row r (lanes >= D repeat row D - 1) from column r + k at step k, wrapping
        // around: the rotated column of every step is computed once, so each product is a
        // gather of the row into registers followed by D shuffle-multiply-adds
        const int lr = lane < D ? lane : D - 1;
        int cidx[32];
#pragma unroll
        for (int k = 0; k < 32; k++) {
            const int c = lr + k;
            cidx[k] = c >= D ? c - D : c;
        }
        int issued = 0, waited = 0;
        if (m0 < tile) {
            if (lane == 0) issue(0, m0);
            issued = 1;
        }
        bool ok = true;
        for (int m = m0, b = 0; m < tile && ok; b++) {
            const int buf = b & 1, cnt = min(nb, tile - m), mn = m + cnt;
            if (mn < tile) {  // the other buffer was last read in batch b - 1, finished by the warp
                if (lane == 0) {
                    tc::fence_async_smem();
                    issue(buf ^ 1, mn);
                }
                issued++;
            }
            Spin spin(spin_limit);
            while (!tc::mbar_try_wait(bars + 8u * (uint32_t)buf, (uint32_t)(b >> 1) & 1u))
                if (!spin.again()) {
                    ok = false;
                    break;
                }
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicExch(&ctl->timeout, 1u);
                v = R(0);
                break;
            }
            waited++;
            const R *stg = stage + (size_t)buf * nb * AS;
            for (int q = 0; q < cnt; q++) {
                const R *Aq = stg + (size_t)q * AS;
                const R *Ar = Aq + lr * D;
                R row[32];
#pragma unroll
                for (int k = 0; k < 32; k++) row[k] = k < D ? Ar[cidx[k]] : R(0);
                R acc[4] = {Aq[DD + lr], R(0), R(0), R(0)};
#pragma unroll
                for (int k = 0; k < 32; k++) {
                    const R vk = __shfl_sync(0xffffffffu, v, k < D ? cidx[k] : 0);
                    if (k < D) acc[k & 3] = fma(row[k], vk, acc[k & 3]);
                }
                v = lane < D ? (acc[0] + acc[1]) + (acc[2] + acc[3]) : R(0);
            }
            __syncwarp();
            m = mn;
        }
        // copies issued but not waited for (after a timeout): let them land before the buffers
        // are reused or the block exits
        if (lane == 0)
            for (int b = waited; b < issued; b++)
                tc::mbar_wait_drain(bars + 8u * (uint32_t)(b & 1), (uint32_t)(b >> 1) & 1u, 1u << 20);
        __syncwarp();
        if (lane < D) carry_out[lane] = v;
    }
    Bar::sync();
}

}  // namespace pm
