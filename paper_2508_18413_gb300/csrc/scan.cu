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
#include <algorithm>
#include <numeric>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"
#include "lookback.cuh"
#include "scan_util.cuh"
#include "scan_rows.cuh"

namespace pm {

namespace {

constexpr int kScanThreads = 256;

__device__ __forceinline__ int smem_idx(int e) { return e + (e >> 5); }  // pad 1 word / 32

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

    if (stats) block_stats(stats, (double)dmax, resets);
    finish_tile(ctl, ntiles);
}

// The row kernel (scan_diag_rows_kernel) is in scan_rows.cuh.

// ==========================================================================================
// Diagonal scan, D <= 32, one register-resident sub-chunk per warp: each lane loads its ROWS
// (a, b, s) elements once, scans its rows in place, and keeps the row prefixes in registers
// through the look-back, so every element crosses HBM exactly once (read a, b, s; write s).
// Small tiles (8 ROWS P timesteps) keep many CTAs resident, which hides the look-back latency.
// ==========================================================================================
template <typename R, typename S, int ROWS>
__global__ void __launch_bounds__(256, (ROWS > 8 || sizeof(R) == 8) ? 2 : 4)
scan_diag_reg_kernel(int T, int D, const S *__restrict__ a, const S *__restrict__ b,
                     R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                     R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl, EvalStats *stats,
                     const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    __shared__ unsigned int s_tile, s_epoch;
    __shared__ R wA[8][32], wB[8][32];   // warp aggregates per channel
    __shared__ R cin[8][32];             // carry into each warp
    __shared__ R tA[32], tB[32], ccar[32];
    const int P = 32 / D, L = P * D;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int WT = ROWS * P;             // timesteps per warp
    const int TT = 8 * WT;
    const unsigned int ntiles = (unsigned int)ceil_div(T, TT);
    const int tile = (int)take_tile(ctl, &s_tile, &s_epoch);
    const unsigned int epoch = s_epoch;
    const bool lane_on = lane < L;
    const int d = lane_on ? lane % D : 0;
    const int tsub = lane_on ? lane / D : 0;
    const int last_lane = (P - 1) * D + d;
    const long long t_base = (long long)tile * TT + (long long)w * WT;

    R ra[ROWS], rb[ROWS], rs[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        const long long t = t_base + (long long)r * P + tsub;
        const bool in = lane_on && t < T;
        const size_t e = (size_t)t * D + d;
        ra[r] = in ? ldg_as<S, R>(a + e) : R(1);
        rb[r] = in ? ldg_as<S, R>(b + e) : R(0);
    }
#pragma unroll
    for (int r = 0; r < ROWS; r++) {  // s is only needed after the look-back
        const long long t = t_base + (long long)r * P + tsub;
        rs[r] = (lane_on && t < T) ? __ldcs(s + (size_t)t * D + d) : R(0);
    }
    R WA = R(1), WB = R(0);
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        for (int off = D; off < L; off <<= 1) {
            const R pa = __shfl_up_sync(0xffffffffu, ra[r], off);
            const R pb = __shfl_up_sync(0xffffffffu, rb[r], off);
            if (lane_on && lane >= off) {
                rb[r] = ra[r] * pb + rb[r];
                ra[r] = ra[r] * pa;
            }
        }
        const R ea = __shfl_sync(0xffffffffu, ra[r], last_lane);
        const R eb = __shfl_sync(0xffffffffu, rb[r], last_lane);
        WB = ea * WB + eb;
        WA = ea * WA;
    }
    if (lane < D) {
        wA[w][lane] = WA;
        wB[w][lane] = WB;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        const int dd = threadIdx.x;
        R TA_ = R(1), TB_ = R(0);
        for (int q = 0; q < 8; q++) {
            TB_ = wA[q][dd] * TB_ + wB[q][dd];
            TA_ = wA[q][dd] * TA_;
        }
        tA[dd] = TA_;
        tB[dd] = TB_;
        if (tile == 0) {
            gincl[dd] = TB_;
        } else {
            gagg[((size_t)tile * 2) * D + dd] = TA_;
            gagg[((size_t)tile * 2 + 1) * D + dd] = TB_;
        }
        ccar[dd] = R(0);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release(flags + tile, make_flag(epoch, tile == 0 ? kFlagIncl : kFlagAgg));
    if (tile > 0) {
        lookback_block64<R>(flags, gagg, gincl, tile, D, epoch, spin_limit, ctl, ccar);
        if (threadIdx.x < D) {
            gincl[(size_t)tile * D + threadIdx.x] = tA[threadIdx.x] * ccar[threadIdx.x] + tB[threadIdx.x];
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) st_release(flags + tile, make_flag(epoch, kFlagIncl));
    }
    if (threadIdx.x < D) {
        const int dd = threadIdx.x;
        R pa = R(1), pb = R(0);
        const R c = ccar[dd];
        for (int q = 0; q < 8; q++) {
            cin[q][dd] = pa * c + pb;
            pb = wA[q][dd] * pb + wB[q][dd];
            pa = wA[q][dd] * pa;
        }
    }
    __syncthreads();
    // rows in order from the carry, from the prefixes held in registers
    R delta = lane_on ? cin[w][d] : R(0);
    R dmax = R(0);
    unsigned int resets = 0;
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        const R dl = ra[r] * delta + rb[r];
        const long long t = t_base + (long long)r * P + tsub;
        if (lane_on && t < T) {
            R sn = rs[r] + dl;
            if (!finite(sn)) {
                sn = s_reset ? s_reset[d] : R(0);
                resets++;
            } else {
                dmax = max(dmax, fabs(dl));
            }
            __stcs(s + (size_t)t * D + d, sn);
        }
        delta = __shfl_sync(0xffffffffu, dl, last_lane);
    }
    if (stats) block_stats(stats, (double)dmax, resets);
    finish_tile(ctl, ntiles);
}

// ==========================================================================================
// Diagonal scan, D <= 32, staged through shared memory by bulk copies.  One thread issues
// cp.async.bulk copies of the tile's a, b and s (one mbarrier; the sub-16-byte tail of a ragged
// last tile is loaded by plain loads), so every element is read from HBM exactly once.  Rows
// are then scanned from shared memory as in the register-resident kernel: pass 1 composes the
// warp aggregates, the block look-back finds the carry, pass 2 recomputes each row's prefix,
// applies the carry and streams s out.  Tiles of about 8K elements keep two or three CTAs
// resident per SM, so one CTA's look-back overlaps another's copies.
// ==========================================================================================
template <typename R, typename S>
__global__ void __launch_bounds__(256)
scan_diag_staged_kernel(int T, int D, int TT, const S *__restrict__ a, const S *__restrict__ b,
                        R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                        R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl,
                        EvalStats *stats, const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ unsigned int s_tile, s_epoch;
    __shared__ R wA[8][32], wB[8][32];
    __shared__ R cin[8][32];
    __shared__ R tA[32], tB[32], ccar[32];
    const int P = 32 / D, L = P * D;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned int ntiles = (unsigned int)ceil_div(T, TT);
    const uint32_t mbar = tc::smem_u32(&s_mbar);
    if (threadIdx.x == 0) {  // initialised before the CTA barrier inside take_tile: no thread
        tc::mbar_init(mbar, 1);  // touches the mbarrier before its initialisation is visible
        tc::fence_barrier_init();
    }
    const int tile = (int)take_tile(ctl, &s_tile, &s_epoch);
    const unsigned int epoch = s_epoch;
    const long long t0 = (long long)tile * TT;
    const int TTv = (int)min((long long)TT, (long long)T - t0);
    const int Ev = TTv * D;
    const size_t E = (size_t)TT * D;
    const size_t ab_region = (E * sizeof(S) + 15) & ~(size_t)15;
    S *sa = reinterpret_cast<S *>(smem_raw);
    S *sbv = reinterpret_cast<S *>(smem_raw + ab_region);
    R *ss = reinterpret_cast<R *>(smem_raw + 2 * ab_region);
    const size_t base = (size_t)t0 * D;
    const uint32_t ab_bytes = (uint32_t)(((size_t)Ev * sizeof(S)) & ~(size_t)15);
    const uint32_t s_bytes = (uint32_t)(((size_t)Ev * sizeof(R)) & ~(size_t)15);
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(mbar, 2 * ab_bytes + s_bytes);
        if (ab_bytes) {
            tc::bulk_g2s(tc::smem_u32(sa), a + base, ab_bytes, mbar);
            tc::bulk_g2s(tc::smem_u32(sbv), b + base, ab_bytes, mbar);
        }
        if (s_bytes) tc::bulk_g2s(tc::smem_u32(ss), s + base, s_bytes, mbar);
    }
    for (int e = (int)(ab_bytes / sizeof(S)) + threadIdx.x; e < Ev; e += 256) {
        sa[e] = a[base + e];
        sbv[e] = b[base + e];
    }
    for (int e = (int)(s_bytes / sizeof(R)) + threadIdx.x; e < Ev; e += 256) ss[e] = s[base + e];
    // the copies complete on their own; the bound only guards against a lost completion
    if (!tc::mbar_wait_drain(mbar, 0, 1u << 20) && threadIdx.x == 0) atomicExch(&ctl->timeout, 1u);
    __syncthreads();

    const bool lane_on = lane < L;
    const int d = lane_on ? lane % D : 0;
    const int tsub = lane_on ? lane / D : 0;
    const int last_lane = (P - 1) * D + d;
    const int RW = TT / (8 * P);  // rows per warp
    const int tw = w * RW * P;    // first local timestep of the warp

    // pass 1: warp aggregates from shared memory
    R WA = R(1), WB = R(0);
#pragma unroll 4
    for (int r = 0; r < RW; r++) {
        const int tl = tw + r * P + tsub;
        const bool in = lane_on && tl < TTv;
        R ra = in ? load_as<S, R>(sa + tl * D + d) : R(1);
        R rb = in ? load_as<S, R>(sbv + tl * D + d) : R(0);
        for (int off = D; off < L; off <<= 1) {
            const R pa = __shfl_up_sync(0xffffffffu, ra, off);
            const R pb = __shfl_up_sync(0xffffffffu, rb, off);
            if (lane_on && lane >= off) {
                rb = ra * pb + rb;
                ra = ra * pa;
            }
        }
        const R ea = __shfl_sync(0xffffffffu, ra, last_lane);
        const R eb = __shfl_sync(0xffffffffu, rb, last_lane);
        WB = ea * WB + eb;
        WA = ea * WA;
    }
    if (lane < D) {
        wA[w][lane] = WA;
        wB[w][lane] = WB;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        const int dd = threadIdx.x;
        R TA_ = R(1), TB_ = R(0);
        for (int q = 0; q < 8; q++) {
            TB_ = wA[q][dd] * TB_ + wB[q][dd];
            TA_ = wA[q][dd] * TA_;
        }
        tA[dd] = TA_;
        tB[dd] = TB_;
        if (tile == 0) {
            gincl[dd] = TB_;
        } else {
            gagg[((size_t)tile * 2) * D + dd] = TA_;
            gagg[((size_t)tile * 2 + 1) * D + dd] = TB_;
        }
        ccar[dd] = R(0);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release(flags + tile, make_flag(epoch, tile == 0 ? kFlagIncl : kFlagAgg));
    if (tile > 0) {
        lookback_block64<R>(flags, gagg, gincl, tile, D, epoch, spin_limit, ctl, ccar);
        if (threadIdx.x < D) {
            gincl[(size_t)tile * D + threadIdx.x] = tA[threadIdx.x] * ccar[threadIdx.x] + tB[threadIdx.x];
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) st_release(flags + tile, make_flag(epoch, kFlagIncl));
    }
    if (threadIdx.x < D) {
        const int dd = threadIdx.x;
        R pa = R(1), pb = R(0);
        const R c = ccar[dd];
        for (int q = 0; q < 8; q++) {
            cin[q][dd] = pa * c + pb;
            pb = wA[q][dd] * pb + wB[q][dd];
            pa = wA[q][dd] * pa;
        }
    }
    __syncthreads();
    // pass 2: rows in order from the carry; s streamed out
    R delta = lane_on ? cin[w][d] : R(0);
    R dmax = R(0);
    unsigned int resets = 0;
#pragma unroll 4
    for (int r = 0; r < RW; r++) {
        const int tl = tw + r * P + tsub;
        const bool in = lane_on && tl < TTv;
        R ra = in ? load_as<S, R>(sa + tl * D + d) : R(1);
        R rb = in ? load_as<S, R>(sbv + tl * D + d) : R(0);
        for (int off = D; off < L; off <<= 1) {
            const R pa = __shfl_up_sync(0xffffffffu, ra, off);
            const R pb = __shfl_up_sync(0xffffffffu, rb, off);
            if (lane_on && lane >= off) {
                rb = ra * pb + rb;
                ra = ra * pa;
            }
        }
        const R dl = ra * delta + rb;
        if (in) {
            const int e = tl * D + d;
            R sn = ss[e] + dl;
            if (!finite(sn)) {
                sn = s_reset ? s_reset[d] : R(0);
                resets++;
            } else {
                dmax = max(dmax, fabs(dl));
            }
            __stcs(s + base + e, sn);
        }
        delta = __shfl_sync(0xffffffffu, dl, last_lane);
    }
    if (stats) block_stats(stats, (double)dmax, resets);
    finish_tile(ctl, ntiles);
}

// ==========================================================================================
// Diagonal scan, D <= 32, persistent and double-buffered: one CTA per SM holds two shared-memory
// tile buffers.  While the CTA scans tile k from one buffer, the bulk copies of the next tile it
// took a ticket for are already filling the other, so every SM keeps a tile's worth of reads in
// flight through its own look-back and compute.  Each element of a, b and s is read from HBM
// once, by a bulk copy (the sub-16-byte tail of a ragged last tile by plain loads).
//
// Within a tile each of the P = 32 / D lane groups of a warp (lane = q D + d) owns a contiguous
// run of M timesteps of channel d, which it composes (pass 1) and later applies (pass 2) one
// timestep at a time in registers; only the P group aggregates of a warp are combined across
// lanes.  The run length satisfies (M - 1) D = 0 mod 64 where the tile size allows, so the P
// groups' shared-memory words fall in distinct banks.
//
// Ordering.  Tickets are taken in increasing order and each CTA processes its tickets in the
// order taken, so the lowest tile without a published aggregate is always the current tile of
// a running CTA that is not waiting: the look-back cannot deadlock on a prefetched tile.
// ==========================================================================================
template <typename R, typename S>
__global__ void __launch_bounds__(256, 1)
scan_diag_pipe_kernel(int T, int D, int M, const S *__restrict__ a, const S *__restrict__ b,
                      R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                      R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl, EvalStats *stats,
                      const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ unsigned int s_first, s_next[2], s_epoch;
    __shared__ R wA[8][32], wB[8][32];
    __shared__ R cin[8][32];
    __shared__ R tA[32], tB[32], ccar[32];
    const int P = 32 / D, L = P * D;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int TT = 8 * P * M;  // timesteps per tile
    const unsigned int ntiles = (unsigned int)ceil_div(T, TT);
    const size_t E = (size_t)TT * D;
    const size_t ab_region = (E * sizeof(S) + 15) & ~(size_t)15;
    const size_t s_region = (E * sizeof(R) + 15) & ~(size_t)15;
    const size_t buf_bytes = 2 * ab_region + s_region;
    const uint32_t mbar0 = tc::smem_u32(&s_mbar[0]);

    // start the bulk copies of `tile` into buffer `bi` (one thread)
    auto issue = [&](unsigned int tile, int bi) {
        const long long t0 = (long long)tile * TT;
        const int Ev = (int)min((long long)TT, (long long)T - t0) * D;
        const size_t base = (size_t)t0 * D;
        unsigned char *buf = smem_raw + (size_t)bi * buf_bytes;
        const uint32_t ab_bytes = (uint32_t)(((size_t)Ev * sizeof(S)) & ~(size_t)15);
        const uint32_t s_bytes = (uint32_t)(((size_t)Ev * sizeof(R)) & ~(size_t)15);
        const uint32_t bar = mbar0 + 8u * (uint32_t)bi;
        tc::mbar_arrive_expect_tx(bar, 2 * ab_bytes + s_bytes);
        if (ab_bytes) {
            tc::bulk_g2s(tc::smem_u32(buf), a + base, ab_bytes, bar);
            tc::bulk_g2s(tc::smem_u32(buf + ab_region), b + base, ab_bytes, bar);
        }
        if (s_bytes) tc::bulk_g2s(tc::smem_u32(buf + 2 * ab_region), s + base, s_bytes, bar);
    };

    if (threadIdx.x == 0) {
        tc::mbar_init(mbar0, 1);
        tc::mbar_init(mbar0 + 8u, 1);
        tc::fence_barrier_init();
        const unsigned int t = atomicAdd(&ctl->ticket, 1u);
        s_first = t;
        s_epoch = *(volatile unsigned int *)&ctl->epoch;
        if (t < ntiles) issue(t, 0);
    }
    __syncthreads();
    const unsigned int epoch = s_epoch;
    const bool lane_on = lane < L;
    const int d = lane_on ? lane % D : 0;
    const int q = lane_on ? lane / D : 0;
    const int last_lane = (P - 1) * D + d;  // lane holding the warp aggregate of channel d
    const int tg = (w * P + q) * M;         // first local timestep of this lane group's run
    R dmax = R(0);
    unsigned int resets = 0;
    unsigned int cur = s_first;
    for (int it = 0; cur < ntiles; it++) {
        const int bi = it & 1;
        const int tile = (int)cur;
        // the other buffer was released by the barrier that ended the previous iteration
        if (threadIdx.x == 0) {
            const unsigned int nx = atomicAdd(&ctl->ticket, 1u);
            s_next[bi] = nx;
            if (nx < ntiles) {
                tc::fence_async_smem();  // earlier generic writes to that buffer (tail loads)
                issue(nx, bi ^ 1);
            }
        }
        const long long t0 = (long long)tile * TT;
        const int TTv = (int)min((long long)TT, (long long)T - t0);
        const int Ev = TTv * D;
        const size_t base = (size_t)t0 * D;
        unsigned char *buf = smem_raw + (size_t)bi * buf_bytes;
        S *sa = reinterpret_cast<S *>(buf);
        S *sbv = reinterpret_cast<S *>(buf + ab_region);
        R *ss = reinterpret_cast<R *>(buf + 2 * ab_region);
        // the copies complete on their own; the bound only guards against a lost completion
        if (!tc::mbar_wait_drain(mbar0 + 8u * (uint32_t)bi, (uint32_t)(it >> 1) & 1u, 1u << 20) &&
            threadIdx.x == 0)
            atomicExch(&ctl->timeout, 1u);
        const int ab_done = (int)((((size_t)Ev * sizeof(S)) & ~(size_t)15) / sizeof(S));
        const int s_done = (int)((((size_t)Ev * sizeof(R)) & ~(size_t)15) / sizeof(R));
        if (ab_done < Ev || s_done < Ev) {  // uniform: only a ragged last tile
            for (int e = ab_done + threadIdx.x; e < Ev; e += 256) {
                sa[e] = a[base + e];
                sbv[e] = b[base + e];
            }
            for (int e = s_done + threadIdx.x; e < Ev; e += 256) ss[e] = s[base + e];
            __syncthreads();
        }
        const int mv = lane_on ? max(0, min(M, TTv - tg)) : 0;  // timesteps of the run in range

        // pass 1: the run's composed map, one timestep at a time
        R GA = R(1), GB = R(0);
#pragma unroll 4
        for (int j = 0; j < mv; j++) {
            const int e = (tg + j) * D + d;
            const R ra = load_as<S, R>(sa + e);
            GB = ra * GB + load_as<S, R>(sbv + e);
            GA = ra * GA;
        }
        // inclusive scan over the P runs of the warp (channel-segmented, later run on the left)
        R IA = GA, IB = GB;
        for (int off = D; off < L; off <<= 1) {
            const R pa = __shfl_up_sync(0xffffffffu, IA, off);
            const R pb = __shfl_up_sync(0xffffffffu, IB, off);
            if (lane_on && lane >= off) {
                IB = IA * pb + IB;
                IA = IA * pa;
            }
        }
        {
            const R ea = __shfl_sync(0xffffffffu, IA, last_lane);
            const R eb = __shfl_sync(0xffffffffu, IB, last_lane);
            if (lane < D) {
                wA[w][lane] = ea;
                wB[w][lane] = eb;
            }
        }
        __syncthreads();
        if (threadIdx.x < D) {
            const int dd = threadIdx.x;
            R TA_ = R(1), TB_ = R(0);
            for (int k = 0; k < 8; k++) {
                TB_ = wA[k][dd] * TB_ + wB[k][dd];
                TA_ = wA[k][dd] * TA_;
            }
            tA[dd] = TA_;
            tB[dd] = TB_;
            if (tile == 0) {
                gincl[dd] = TB_;
            } else {
                gagg[((size_t)tile * 2) * D + dd] = TA_;
                gagg[((size_t)tile * 2 + 1) * D + dd] = TB_;
            }
            ccar[dd] = R(0);
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) st_release(flags + tile, make_flag(epoch, tile == 0 ? kFlagIncl : kFlagAgg));
        if (tile > 0) {
            lookback_block64<R>(flags, gagg, gincl, tile, D, epoch, spin_limit, ctl, ccar);
            if (threadIdx.x < D) {
                gincl[(size_t)tile * D + threadIdx.x] = tA[threadIdx.x] * ccar[threadIdx.x] + tB[threadIdx.x];
                __threadfence();
            }
            __syncthreads();
            if (threadIdx.x == 0) st_release(flags + tile, make_flag(epoch, kFlagIncl));
        }
        if (threadIdx.x < D) {
            const int dd = threadIdx.x;
            R pa = R(1), pb = R(0);
            const R c = ccar[dd];
            for (int k = 0; k < 8; k++) {
                cin[k][dd] = pa * c + pb;
                pb = wA[k][dd] * pb + wB[k][dd];
                pa = wA[k][dd] * pa;
            }
        }
        __syncthreads();
        // pass 2: the carry into the run (the end of the previous run of the warp), then the
        // run's timesteps in order; s streamed out
        const R cw = lane_on ? cin[w][d] : R(0);
        R delta = __shfl_up_sync(0xffffffffu, IA * cw + IB, D);
        if (lane < D) delta = cw;
#pragma unroll 4
        for (int j = 0; j < mv; j++) {
            const int e = (tg + j) * D + d;
            delta = load_as<S, R>(sa + e) * delta + load_as<S, R>(sbv + e);
            R sn = ss[e] + delta;
            if (!finite(sn)) {
                sn = s_reset ? s_reset[d] : R(0);
                resets++;
            } else {
                dmax = max(dmax, fabs(delta));
            }
            __stcs(s + base + e, sn);
        }
        __syncthreads();  // this buffer is free for the copy issued next iteration
        cur = s_next[bi];
    }
    if (stats) block_stats(stats, (double)dmax, resets);
    exit_persistent(ctl);
}

// Timesteps per tile of the staged kernel: about 8K elements (4K in FP64), a multiple of the
// 8 P timesteps of a CTA's rows (P = 32 / D), and small enough to give every SM two tiles.
static int staged_tile(int T, int D, int elem_bytes) {
    const int P = 32 / D, unit = 8 * P;
    const int target = (elem_bytes >= 8 ? 4096 : 8192) / D;
    int tt = std::max(unit, target / unit * unit);
    const int spread = ceil_div(ceil_div(T, 2 * 152), unit) * unit;
    return std::max(unit, std::min(tt, spread));
}

static size_t staged_smem(int TT, int D, int rbytes, int sbytes) {
    const size_t E = (size_t)TT * D;
    return 2 * ((E * sbytes + 15) & ~(size_t)15) + E * rbytes;
}

// CTAs per SM of the pipelined kernel: PMCMC_PIPE_CTAS = 1 or 2 (read at every launch; default
// 1).  With two, each CTA holds half the shared memory (smaller tiles) and one CTA's barrier
// and look-back latency overlaps the other's work.
static int pipe_ctas() {
    const char *e = getenv("PMCMC_PIPE_CTAS");
    return (e && e[0] == '2') ? 2 : 1;
}

// Run length M of the pipelined kernel (its tile is 8 P M timesteps): two tile buffers of a, b
// and s within about 216 KB of shared memory per SM (200 KB with two CTAs, each also holding its
// static shared memory), at least two tiles per CTA where T allows,
// and M - 1 a multiple of 32 / gcd(D, 32) (the P runs of a warp then start in distinct banks)
// unless that would halve the run.
static int pipe_run(int T, int D, int sbytes, int rbytes, int ctas) {
    const int P = 32 / D;
    const int per_elem = 2 * sbytes + rbytes;
    const int buf = ctas == 1 ? 108 * 1024 : 50 * 1024;  // two buffers (+ static) per CTA
    const int m_max = std::max(1, buf / (8 * P * D * per_elem));
    const int spread = std::max(1, ceil_div(T, 2 * 152 * ctas * 8 * P));
    const int cap = std::min(m_max, spread);
    if (P == 1) return cap;
    const int c = 32 / std::gcd(D, 32);
    const int m = (cap - 1) / c * c + 1;
    return 2 * m >= cap ? m : cap;
}

static size_t pipe_smem(int M, int D, int sbytes, int rbytes) {
    const size_t E = (size_t)8 * (32 / D) * M * D;
    return 2 * (2 * ((E * sbytes + 15) & ~(size_t)15) + ((E * rbytes + 15) & ~(size_t)15));
}

// Kernel choice for D <= 32.  By default the pipelined kernel in a middle range of T D and the
// register-resident kernels otherwise: for 2^21 < T D <= 3 * 2^22 elements in general
// (measured on GB300, D = 2, 8, 25: the pipelined kernel runs 1.5-2x faster there than the
// generic row kernel, whose tiles are either small or few per SM, and slower above, where its
// one tile in flight per SM leaves the look-back latency exposed), and for 2^20 <= T D <= 2^22
// (3 * 2^21 with bfloat16 pairs) where the row kernel has D fixed at compile time (FP32
// iterates, D a power of two).  PMCMC_SCAN_KERNEL=rows, staged, pipe or cluster forces a kernel
// (read at every launch, so a process can compare them).
static int scan_kernel_choice(long long elems, int D, bool f64, int storage) {
    const char *e = getenv("PMCMC_SCAN_KERNEL");
    if (e && strcmp(e, "rows") == 0) return 0;
    if (e && strcmp(e, "staged") == 0) return 1;
    if (e && strcmp(e, "pipe") == 0) return 2;
    if (e && strcmp(e, "cluster") == 0) return 3;
    // FP32 iterates with D a power of two, where the row kernel has D fixed at compile time
    // (measured on GB300, D = 8: the pipelined kernel is faster from 2^20 to 2^22 elements,
    // 3 2^21 with bfloat16 pairs; the row kernel from 3 2^21 (FP32) and 3 2^22 (bfloat16))
    const char *dc = getenv("PMCMC_SCAN_DCONST");
    if (!f64 && (D & (D - 1)) == 0 && !(dc && dc[0] == '0'))
        return (elems >= (1ll << 20) && elems <= (storage == 1 ? 3ll << 21 : 1ll << 22)) ? 2 : 0;
    return (elems > (1ll << 21) && elems <= 3ll * (1ll << 22)) ? 2 : 0;
}

int diag_scan_tile(int T, int D, int elem_bytes) {
    if (D <= 32)  // the smallest tile of the kernels that may run sizes the workspace
        return std::min({diag_scan_tile_rows(T, D), staged_tile(T, D, elem_bytes),
                         8 * (32 / D) * pipe_run(T, D, elem_bytes, elem_bytes, 2),
                         diag_scan_tile_cluster(D, 4)});
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
    cudaError_t e = ensure_dyn_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<ntiles, kScanThreads, sm, st>>>(T, D, TT, (const S *)a, (const S *)b, (R *)s,
                                        (const R *)s_reset, w.flags, (R *)w.agg, (R *)w.incl,
                                        w.ctl, stats, skip, spin);
    return cudaGetLastError();
}

// Tile shape of the register-resident scan: rows per sub-chunk (8 or 16) and sub-chunks per
// warp.  scan_shape_override() lets the autotuner (and measurements) fix a shape.
static int g_shape_rows = 0, g_shape_nsub = 0;
void scan_shape_override(int rows, int nsub) {
    g_shape_rows = rows;
    g_shape_nsub = nsub;
}

static void diag_shape(int T, int D, int *rows, int *nsub) {
    {  // PMCMC_SCAN_SHAPE="rows,nsub" fixes the shape (measurements, tests); read at every call
        const char *e = getenv("PMCMC_SCAN_SHAPE");
        int r = 0, n = 0;
        if (e && sscanf(e, "%d,%d", &r, &n) == 2 && (r == 8 || r == 16) && n >= 1 && n <= 64) {
            *rows = r;
            *nsub = n;
            return;
        }
    }
    *rows = g_shape_rows > 0 ? g_shape_rows : 8;
    if (g_shape_nsub > 0) {
        *nsub = g_shape_nsub;
        return;
    }
    // measured on GB300 (2^26..2^28 elements): larger tiles amortise the fixed per-tile latency
    // (ticket, fences, look-back) up to ~32 sub-chunks, as long as the tiles still keep every
    // SM busy several times over: 32 or 16 sub-chunks with at least 8 tiles per SM, else up to
    // 8 with at least 4 tiles per SM (at 2^24 elements 8 sub-chunks ran 4-10% faster than 4)
    const int P = 32 / D;
    *nsub = 0;
    for (int n : {32, 16, 8, 4, 2, 1})
        if (ceil_div(T, 8 * *rows * n * P) >= (n >= 16 ? 8 : 4) * 152) {
            *nsub = n;
            break;
        }
    if (*nsub == 0) {
        *nsub = 1;
        for (int n : {16, 8, 4, 2, 1})
            if (ceil_div(T, 8 * *rows * n * P) >= 2 * 152) {
                *nsub = n;
                break;
            }
    }
}

// CTAs of `kernel` (block of `threads`, `dyn_smem` bytes of dynamic shared memory) resident on
// the device at once, cached per kernel and shared-memory size.
template <class K>
static int resident_ctas(K kernel, int threads, size_t dyn_smem = 0) {
    static const void *keys[32] = {};
    static size_t smems[32] = {};
    static int vals[32] = {};
    static int n = 0;
    const void *key = reinterpret_cast<const void *>(kernel);
    for (int i = 0; i < n; i++)
        if (keys[i] == key && smems[i] == dyn_smem) return vals[i];
    int per_sm = 1, dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int v = per_sm * sms;
    if (n < 32) {
        keys[n] = key;
        smems[n] = dyn_smem;
        vals[n++] = v;
    }
    return v;
}

template <typename R, typename S>
static cudaError_t run_scan_rows(int T, int D, const void *a, const void *b, void *s,
                                 const void *s_reset, const ScanWork &w, EvalStats *stats,
                                 const int *skip, unsigned int spin, cudaStream_t st) {
    int rows, nsub;
    diag_shape(T, D, &rows, &nsub);
    const int ntiles = ceil_div(T, 8 * rows * nsub * (32 / D));
    if (ntiles > w.max_tiles) return cudaErrorInvalidValue;
    if (nsub == 1) {  // one sub-chunk: the register-resident single-read kernel
        if (rows == 16) {
            prefer_shared(scan_diag_reg_kernel<R, S, 16>);
            scan_diag_reg_kernel<R, S, 16><<<ntiles, 256, 0, st>>>(
                T, D, (const S *)a, (const S *)b, (R *)s, (const R *)s_reset, w.flags, (R *)w.agg,
                (R *)w.incl, w.ctl, stats, skip, spin);
        } else {
            prefer_shared(scan_diag_reg_kernel<R, S, 8>);
            scan_diag_reg_kernel<R, S, 8><<<ntiles, 256, 0, st>>>(
                T, D, (const S *)a, (const S *)b, (R *)s, (const R *)s_reset, w.flags, (R *)w.agg,
                (R *)w.incl, w.ctl, stats, skip, spin);
        }
        return cudaGetLastError();
    }
    // persistent grid: at most the CTAs that can be resident at once
    // D a power of two (1 .. 32): the instance with D fixed at compile time (its index arithmetic
    // folds away; measured 4-23% faster on GB300); PMCMC_SCAN_DCONST=0 keeps the generic one
    const char *dc = getenv("PMCMC_SCAN_DCONST");
    if (rows == 8 && (D & (D - 1)) == 0 && !(dc && dc[0] == '0')) {
        const int kind = sizeof(R) == 8 ? 2 : (sizeof(S) == 2 ? 1 : 0);
        return launch_scan_rows_dconst(kind, T, D, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
    }
    if (rows == 16) {
        auto k = scan_diag_rows_kernel<R, S, 16>;
        prefer_shared(k);
        k<<<std::min(ntiles, resident_ctas(k, 256)), 256, 0, st>>>(
            T, D, nsub, (const S *)a, (const S *)b, (R *)s, (const R *)s_reset, w.flags,
            (R *)w.agg, (R *)w.incl, w.ctl, stats, skip, spin);
    } else {
        auto k = scan_diag_rows_kernel<R, S, 8>;
        prefer_shared(k);
        k<<<std::min(ntiles, resident_ctas(k, 256)), 256, 0, st>>>(
            T, D, nsub, (const S *)a, (const S *)b, (R *)s, (const R *)s_reset, w.flags,
            (R *)w.agg, (R *)w.incl, w.ctl, stats, skip, spin);
    }
    return cudaGetLastError();
}

int diag_scan_tile_rows(int T, int D) {
    int rows, nsub;
    diag_shape(T, D, &rows, &nsub);
    return 8 * rows * nsub * (32 / D);
}

template <typename R, typename S>
static cudaError_t run_scan_staged(int T, int D, const void *a, const void *b, void *s,
                                   const void *s_reset, const ScanWork &w, EvalStats *stats,
                                   const int *skip, unsigned int spin, cudaStream_t st) {
    const int TT = staged_tile(T, D, sizeof(R));
    const int ntiles = ceil_div(T, TT);
    if (ntiles > w.max_tiles) return cudaErrorInvalidValue;
    const size_t sm = staged_smem(TT, D, sizeof(R), sizeof(S));
    auto k = scan_diag_staged_kernel<R, S>;
    cudaError_t e = ensure_dyn_smem(k, sm);
    if (e != cudaSuccess) return e;
    prefer_shared(k);
    k<<<ntiles, 256, sm, st>>>(T, D, TT, (const S *)a, (const S *)b, (R *)s, (const R *)s_reset,
                               w.flags, (R *)w.agg, (R *)w.incl, w.ctl, stats, skip, spin);
    return cudaGetLastError();
}

template <typename R, typename S>
static cudaError_t run_scan_pipe(int T, int D, const void *a, const void *b, void *s,
                                 const void *s_reset, const ScanWork &w, EvalStats *stats,
                                 const int *skip, unsigned int spin, cudaStream_t st) {
    const int M = pipe_run(T, D, sizeof(S), sizeof(R), pipe_ctas());
    const int ntiles = ceil_div(T, 8 * (32 / D) * M);
    if (ntiles > w.max_tiles) return cudaErrorInvalidValue;
    const size_t sm = pipe_smem(M, D, sizeof(S), sizeof(R));
    auto k = scan_diag_pipe_kernel<R, S>;
    cudaError_t e = ensure_dyn_smem(k, sm);
    if (e != cudaSuccess) return e;
    // persistent: every CTA must be resident at once (the look-back waits on other CTAs)
    k<<<std::min(ntiles, resident_ctas(k, 256, sm)), 256, sm, st>>>(
        T, D, M, (const S *)a, (const S *)b, (R *)s, (const R *)s_reset, w.flags, (R *)w.agg,
        (R *)w.incl, w.ctl, stats, skip, spin);
    return cudaGetLastError();
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cudaError_t launch_scan_diag(bool f64, int storage, int T, int D, int tile_t, const void *a,
                             const void *b, void *s, const void *s_reset, const ScanWork &w,
                             EvalStats *stats, const int *skip, unsigned int spin_limit,
                             cudaStream_t st) {
    const int choice = D <= 32 ? scan_kernel_choice((long long)T * D, D, f64, storage) : 0;
    if (D <= 32 && choice == 3 && !f64 && aligned16(a) && aligned16(b) && aligned16(s))
        return launch_scan_diag_cluster(storage, T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    if (D <= 32 && choice == 2 && aligned16(a) && aligned16(b) && aligned16(s)) {
        if (f64) return run_scan_pipe<double, double>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
        if (storage == 1)
            return run_scan_pipe<float, __nv_bfloat16>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
        return run_scan_pipe<float, float>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    }
    if (D <= 32 && choice == 1 && aligned16(a) && aligned16(b) && aligned16(s)) {
        if (f64) return run_scan_staged<double, double>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
        if (storage == 1)
            return run_scan_staged<float, __nv_bfloat16>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
        return run_scan_staged<float, float>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    }
    if (D <= 32) {
        if (f64) return run_scan_rows<double, double>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
        if (storage == 1)
            return run_scan_rows<float, __nv_bfloat16>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
        return run_scan_rows<float, float>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    }
    if (ceil_div(T, tile_t) > w.max_tiles) return cudaErrorInvalidValue;
    if (f64) return run_scan_diag<double, double>(T, D, tile_t, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    if (storage == 1)
        return run_scan_diag<float, __nv_bfloat16>(T, D, tile_t, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    return run_scan_diag<float, float>(T, D, tile_t, a, b, s, s_reset, w, stats, skip, spin_limit, st);
}

// What launch_scan_diag runs for (T, D) with 16-byte-aligned a, b and s, computed from the same
// helpers without device work: the kernel (ScanPlanKernel), its timesteps per tile and the
// tiles of the launch.
void plan_scan_diag(bool f64, int storage, int T, int D, int *kernel, int *tile, int *tiles) {
    const int rb = f64 ? 8 : 4, sbytes = f64 ? 8 : (storage == 1 ? 2 : 4);
    int k = kPlanDiagWide, tt = 0;
    if (D > 32) {
        tt = diag_scan_tile(T, D, rb);
    } else {
        const int choice = scan_kernel_choice((long long)T * D, D, f64, storage);
        const int P = 32 / D;
        if (choice == 3 && !f64) {
            k = kPlanCluster;
            tt = diag_scan_tile_cluster(D, sbytes);
        } else if (choice == 2) {
            k = kPlanPipe;
            tt = 8 * P * pipe_run(T, D, sbytes, rb, pipe_ctas());
        } else if (choice == 1) {
            k = kPlanStaged;
            tt = staged_tile(T, D, rb);
        } else {
            int rows, nsub;
            diag_shape(T, D, &rows, &nsub);
            tt = 8 * rows * nsub * P;
            const char *dc = getenv("PMCMC_SCAN_DCONST");
            if (nsub == 1)
                k = kPlanRegister;
            else if (rows == 8 && (D & (D - 1)) == 0 && !(dc && dc[0] == '0'))
                k = kPlanRowsConstD;
            else
                k = kPlanRows;
        }
    }
    *kernel = k;
    *tile = tt;
    *tiles = ceil_div(T, tt);
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

// ==========================================================================================
// Dense scan for D <= 4: one timestep per thread, the affine element (A, b) in registers.
// Warp shuffle scan, block combine over 8 warps, one look-back per 256-step tile.
// ==========================================================================================
template <typename R, int DM>
struct Aff {
    R A[DM][DM], b[DM];
};

// (later) o (earlier): (A2 A1, A2 b1 + b2)
template <typename R, int DM>
__device__ __forceinline__ Aff<R, DM> compose(const Aff<R, DM> &l, const Aff<R, DM> &e, int D) {
    Aff<R, DM> o;
#pragma unroll
    for (int i = 0; i < DM; i++) {
        R acc = l.b[i];
#pragma unroll
        for (int k = 0; k < DM; k++) acc += l.A[i][k] * e.b[k];
        o.b[i] = acc;
#pragma unroll
        for (int j = 0; j < DM; j++) {
            R m = R(0);
#pragma unroll
            for (int k = 0; k < DM; k++) m += l.A[i][k] * e.A[k][j];
            o.A[i][j] = m;
        }
    }
    (void)D;
    return o;
}

template <typename R, int DM>
__device__ __forceinline__ Aff<R, DM> shfl_up_aff(const Aff<R, DM> &x, int off) {
    Aff<R, DM> o;
#pragma unroll
    for (int i = 0; i < DM; i++) {
        o.b[i] = __shfl_up_sync(0xffffffffu, x.b[i], off);
#pragma unroll
        for (int j = 0; j < DM; j++) o.A[i][j] = __shfl_up_sync(0xffffffffu, x.A[i][j], off);
    }
    return o;
}

template <typename R, int DM>
__global__ void __launch_bounds__(256)
scan_dense_small_kernel(int T, int D, const R *__restrict__ a, const R *__restrict__ b,
                        R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                        R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl,
                        EvalStats *stats, const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    __shared__ unsigned int s_tile, s_epoch;
    __shared__ Aff<R, DM> wagg[8];
    __shared__ R wcar[8][DM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned int ntiles = (unsigned int)ceil_div(T, 256);
    const int tile = (int)take_tile(ctl, &s_tile, &s_epoch);
    const unsigned int epoch = s_epoch;
    const int t = tile * 256 + threadIdx.x;
    const bool in = t < T;
    const int DD = D * D;
    Aff<R, DM> x;
#pragma unroll
    for (int i = 0; i < DM; i++) {
        x.b[i] = (in && i < D) ? b[(size_t)t * D + i] : R(0);
#pragma unroll
        for (int j = 0; j < DM; j++)
            x.A[i][j] = (in && i < D && j < D) ? a[(size_t)t * DD + i * D + j] : (i == j ? R(1) : R(0));
    }
    // warp inclusive scan
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Aff<R, DM> p = shfl_up_aff<R, DM>(x, off);
        if (lane >= off) x = compose<R, DM>(x, p, D);
    }
    if (lane == 31) wagg[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        // warp prefixes, tile aggregate, publish, look back, carries into the warps
        Aff<R, DM> acc = wagg[0];
        for (int q = 1; q < 8; q++) acc = compose<R, DM>(wagg[q], acc, D);
        R c[DM];
#pragma unroll
        for (int i = 0; i < DM; i++) c[i] = R(0);
        if (tile == 0) {
            for (int i = 0; i < D; i++) gincl[i] = acc.b[i];
            __threadfence();
            st_release(flags, make_flag(epoch, kFlagIncl));
        } else {
            const size_t AGG = (size_t)DD + D;
            for (int i = 0; i < D; i++) {
                for (int j = 0; j < D; j++) gagg[(size_t)tile * AGG + i * D + j] = acc.A[i][j];
                gagg[(size_t)tile * AGG + DD + i] = acc.b[i];
            }
            __threadfence();
            st_release(flags + tile, make_flag(epoch, kFlagAgg));
            int jj = tile - 1;
            for (; jj >= 0; jj--) {
                unsigned int st = wait_flag(flags, jj, epoch, spin_limit, ctl);
                if (st == kFlagIncl || st == 0) break;
            }
            if (jj >= 0) {
                unsigned int st = ld_acquire(flags + jj);
                if ((st & 3u) == kFlagIncl && (st >> 2) == (epoch & 0x3fffffffu))
                    for (int i = 0; i < D; i++) c[i] = gincl[(size_t)jj * D + i];
            }
            for (int m = max(jj + 1, 0); m < tile; m++) {
                const R *Am = gagg + (size_t)m * AGG;
                R nc[DM];
                for (int i = 0; i < D; i++) {
                    R v = Am[DD + i];
                    for (int k = 0; k < D; k++) v += Am[i * D + k] * c[k];
                    nc[i] = v;
                }
                for (int i = 0; i < D; i++) c[i] = nc[i];
            }
            for (int i = 0; i < D; i++) {
                R v = acc.b[i];
                for (int k = 0; k < D; k++) v += acc.A[i][k] * c[k];
                gincl[(size_t)tile * D + i] = v;
            }
            __threadfence();
            st_release(flags + tile, make_flag(epoch, kFlagIncl));
        }
        // carry into warp q = (warps < q) applied to c
        for (int q = 0; q < 8; q++) {
            for (int i = 0; i < DM; i++) wcar[q][i] = c[i];
            R nc[DM];
            for (int i = 0; i < D; i++) {
                R v = wagg[q].b[i];
                for (int k = 0; k < D; k++) v += wagg[q].A[i][k] * c[k];
                nc[i] = v;
            }
            for (int i = 0; i < D; i++) c[i] = nc[i];
        }
    }
    __syncthreads();
    R dmax = R(0);
    unsigned int resets = 0;
    if (in) {
#pragma unroll
        for (int i = 0; i < DM; i++) {
            if (i >= D) continue;
            R dl = x.b[i];
#pragma unroll
            for (int k = 0; k < DM; k++) dl += x.A[i][k] * wcar[w][k];
            R sn = s[(size_t)t * D + i] + dl;
            if (!finite(sn)) {
                sn = s_reset ? s_reset[i] : R(0);
                resets++;
            } else {
                dmax = max(dmax, fabs(dl));
            }
            s[(size_t)t * D + i] = sn;
        }
    }
    if (stats) block_stats(stats, (double)dmax, resets);
    finish_tile(ctl, ntiles);
}

int dense_scan_chunk(int T, int D) {
    if (D <= 4) return 256;  // one timestep per thread, 256 per tile
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
    if (D <= 4) {
        if (chunk != 256) return cudaErrorInvalidValue;
#define PM_DS(R_, DM_)                                                                           \
    prefer_shared(scan_dense_small_kernel<R_, DM_>);                                           \
    scan_dense_small_kernel<R_, DM_><<<ceil_div(T, 256), 256, 0, st>>>(                        \
        T, D, (const R_ *)a, (const R_ *)b, (R_ *)s, (const R_ *)s_reset, w.flags, (R_ *)w.agg, \
        (R_ *)w.incl, w.ctl, stats, skip, spin_limit);                                         \
    return cudaGetLastError();
        if (f64) {
            if (D <= 2) { PM_DS(double, 2) }
            PM_DS(double, 4)
        } else {
            if (D <= 2) { PM_DS(float, 2) }
            PM_DS(float, 4)
        }
#undef PM_DS
    }
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
