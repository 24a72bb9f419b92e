// Device helpers shared by the persistent scan kernels: tile tickets, the per-launch reset of the
// ticket counter and epoch, and the block-wide reduction of the scan statistics.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace pm {

namespace {

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

// Block-wide reduction of the scan statistics: one atomic per CTA (same-address atomics from
// every warp of every tile serialise in L2).  Called by all threads of the CTA.
__device__ __forceinline__ void block_stats(EvalStats *stats, double dmax, unsigned int resets) {
    __shared__ double s_dm[32];
    __shared__ unsigned int s_rs[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double dm = warp_max(dmax);
    unsigned int rs = warp_sum(resets);
    if (lane == 0) {
        s_dm[w] = dm;
        s_rs[w] = rs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; i++) {
            dm = fmax(dm, s_dm[i]);
            rs += s_rs[i];
        }
        if (dm > 0) atomic_max_d(&stats->dmax, dm);
        if (rs) atomicAdd(&stats->resets, (unsigned long long)rs);
    }
}

// Exit of a persistent scan kernel: every CTA has taken its last (out-of-range) ticket before it
// counts itself out, so the last CTA to leave can reset the ticket and advance the epoch with
// no CTA left that could take another ticket.
__device__ __forceinline__ void exit_persistent(ScanCtl *ctl) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int e = atomicAdd(&ctl->done, 1u);
        if (e == gridDim.x - 1) {
            ctl->ticket = 0;
            ctl->done = 0;
            ctl->epoch = ctl->epoch + 1u;
            __threadfence();
        }
    }
}

}  // namespace

}  // namespace pm
