// The row kernel of the diagonal scan (D <= 32), shared by scan.cu (D known at run time) and
// scan_rows_dc.cu (D a compile-time constant, the powers of two up to 32).
#pragma once

#include "common.cuh"
#include "internal.h"
#include "lookback.cuh"
#include "scan_util.cuh"

namespace pm {

// ==========================================================================================
// Diagonal scan, D <= 32, register resident.  A row is 32 lanes holding P = 32 / D consecutive
// timesteps of all D channels (L = P D contiguous elements, coalesced).  Each warp owns ROWS
// rows; a CTA (8 warps) owns a tile of 8 ROWS P timesteps.
//   1. every lane loads its ROWS (a, b, s) elements (all loads in flight at once);
//   2. each row is scanned across lanes with a channel-segmented shuffle scan (offsets
//      D, 2D, 4D, ...); the row aggregate of channel d sits in lane (P - 1) D + d;
//   3. rows are composed in order into the warp aggregate, warps into the tile aggregate;
//   4. the tile aggregate is published and the carry found by the bounded look-back;
//   5. rows are applied in order from the carry and s is stored.
// ==========================================================================================
template <typename R, typename S, int ROWS, int DC = 0>
__global__ void __launch_bounds__(256, (ROWS > 8 ? 2 : 4))
scan_diag_rows_kernel(int T, int D_, int NSUB, const S *__restrict__ a, const S *__restrict__ b,
                      R *__restrict__ s, const R *__restrict__ s_reset, unsigned int *flags,
                      R *__restrict__ gagg, R *__restrict__ gincl, ScanCtl *ctl, EvalStats *stats,
                      const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    const int D = DC > 0 ? DC : D_;  // channels (a compile-time constant where DC > 0)
    __shared__ unsigned int s_tile, s_epoch;
    __shared__ R wA[8][32], wB[8][32];   // warp aggregates per channel
    __shared__ R cin[8][32];             // carry into each warp
    const int P = 32 / D, L = P * D;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int WT = NSUB * ROWS * P;      // timesteps per warp (a contiguous chunk)
    const int TT = 8 * WT;
    const unsigned int ntiles = (unsigned int)ceil_div(T, TT);
    const bool lane_on = lane < L;
    const int d = lane_on ? lane % D : 0;
    const int tsub = lane_on ? lane / D : 0;
    const int last_lane = (P - 1) * D + d;  // lane holding the row end of channel d
    R dmax = R(0);
    unsigned int resets = 0;
    // persistent: the CTA takes tiles in ticket order until they run out
    for (;;) {
    const int tile = (int)take_tile(ctl, &s_tile, &s_epoch);
    if (tile >= (int)ntiles) break;
    const unsigned int epoch = s_epoch;
    const long long t_warp = (long long)tile * TT + (long long)w * WT;

    // pass 1: the warp aggregate over its chunk (a, b only)
    R WA = R(1), WB = R(0);
    for (int sub = 0; sub < NSUB; sub++) {
        const long long t_base = t_warp + (long long)sub * ROWS * P;
        R ra[ROWS], rb[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const long long t = t_base + (long long)r * P + tsub;
            const bool in = lane_on && t < T;
            const size_t e = (size_t)t * D + d;
            ra[r] = in ? ldg_as<S, R>(a + e) : R(1);
            rb[r] = in ? ldg_as<S, R>(b + e) : R(0);
        }
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
    }
    if (lane < D) {
        wA[w][lane] = WA;
        wB[w][lane] = WB;
    }
    __syncthreads();
    // tile aggregate, publish, block-wide look-back, carries into the warps
    __shared__ R tA[32], tB[32], ccar[32];
    if (threadIdx.x < D) {
        const int dd = threadIdx.x;
        R TA = R(1), TB = R(0);
        for (int q = 0; q < 8; q++) {
            TB = wA[q][dd] * TB + wB[q][dd];
            TA = wA[q][dd] * TA;
        }
        tA[dd] = TA;
        tB[dd] = TB;
        if (tile == 0) {
            gincl[dd] = TB;
        } else {
            gagg[((size_t)tile * 2) * D + dd] = TA;
            gagg[((size_t)tile * 2 + 1) * D + dd] = TB;
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
    // pass 2: re-read the chunk (a, b from L2), apply rows in order from the carry
    R delta = lane_on ? cin[w][d] : R(0);
    for (int sub = 0; sub < NSUB; sub++) {
        const long long t_base = t_warp + (long long)sub * ROWS * P;
        R ra[ROWS], rb[ROWS], rs[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const long long t = t_base + (long long)r * P + tsub;
            const bool in = lane_on && t < T;
            const size_t e = (size_t)t * D + d;
            ra[r] = in ? ldg_as<S, R>(a + e) : R(1);
            rb[r] = in ? ldg_as<S, R>(b + e) : R(0);
            rs[r] = in ? __ldcs(s + e) : R(0);
        }
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
            const R dl = ra[r] * delta + rb[r];
            const long long t = t_base + (long long)r * P + tsub;
            if (lane_on && t < T) {
                const size_t e = (size_t)t * D + d;
                R sn = rs[r] + dl;
                if (!finite(sn)) {
                    sn = s_reset ? s_reset[d] : R(0);
                    resets++;
                } else {
                    dmax = max(dmax, fabs(dl));
                }
                __stcs(s + e, sn);
            }
            delta = __shfl_sync(0xffffffffu, dl, last_lane);
        }
    }
    __syncthreads();  // shared arrays are reused by the next tile
    }
    if (stats) block_stats(stats, (double)dmax, resets);
    exit_persistent(ctl);
}


}  // namespace pm
