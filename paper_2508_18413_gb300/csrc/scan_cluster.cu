// Diagonal scan (Eq. 3 with a diagonal J_t, as in quasi-DEER), D <= 32, for chains of many
// millions of elements: thread-block clusters share one look-back tile.
//
// The single-pass look-back scan needs a tile large enough that the GPU publishes few tiles per
// microsecond (each look-back round costs two L2 round trips for a window of 32 predecessors),
// while a tile read once must stay on chip between its aggregate and its carry.  Here a tile is
// spread over a cluster of CL CTAs (one per SM): CTA rank r holds sub-tile r of every cluster
// tile in shared memory, the cluster's aggregate is composed in rank 0 through distributed
// shared memory, and one look-back per cluster tile finds its carry.  Each CTA keeps NS sub-tile
// slots: while the look-back of tile k is in flight, its compute warps scan tile k + 1 and the
// bulk copies of later tiles land.  Measured on GB300 it is nevertheless slower than the row
// kernel (28% against 49-52% of HBM at 2^26-2^28 elements): each tile's carry waits for the
// aggregates of the tiles published in the same wave, each ~2.6 us after its cluster aggregate,
// and four slots leave room for only two tiles between pass 1 and pass 2.  It is an option
// (PMCMC_SCAN_KERNEL=cluster), not a default.
//
// Roles (480 threads per CTA):
//   warps 0-7   compute: pass 1 (each lane group composes a run of M timesteps of one channel),
//               the CTA aggregate (sent to rank 0), and LAG tiles later pass 2 (the run applied
//               from its carry, read from rank 0; s written back);
//   warp 8      producer: rank 0 takes the cluster's tickets and hands each to every rank (one
//               lane per rank); every rank copies its sub-tile of a, b, s into a free slot
//               (cp.async.bulk);
//   warps 9-10  (rank 0) publishers, alternating tiles: compose the cluster aggregate and
//               publish it for the look-backs of later tiles;
//   warps 11-14 (rank 0) walkers, one tile in four each: walk the predecessors' flags, leave
//               each rank's carry in rank 0's shared memory, signal the ranks (one lane per
//               rank), publish the inclusive value.
// The fences that publish a value to the GPU take about a microsecond each, so publication and
// look-back run in warps of their own, several tiles at a time.
// Every wait is bounded; a wait that runs out records the timeout, and every role then leaves
// its loop (copies in flight are drained first).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "common.cuh"
#include "internal.h"
#include "lookback.cuh"
#include "scan_util.cuh"
#include "tc.cuh"

namespace pm {

namespace {

constexpr int kCompute = 256;             // compute threads (8 warps)
constexpr int kProducerWarp = 8;
constexpr int kPublisherWarp = 9, kPublishers = 2;
constexpr int kWalkerWarp = 11, kWalkers = 4;
constexpr int kThreads = 32 * (kWalkerWarp + kWalkers);  // 480
constexpr int kMaxCl = 8;               // largest cluster size supported

// ---- cluster primitives --------------------------------------------------------------------
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the variable at local shared address `a` in CTA `rank`
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_st_u32(uint32_t a, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st_f32(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ float cl_ld_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cl_fence() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
// arrive on the mbarrier at shared::cluster address `bar` (any CTA of the cluster)
__device__ __forceinline__ void cl_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
// one poll of a local mbarrier whose arrivals may come from other CTAs of the cluster
__device__ __forceinline__ bool cl_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(tc::kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void compute_bar() {  // the 256 compute threads
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

// Bounded wait (cluster-scope acquire).  Gives up after `limit` polls or once *abort is raised;
// the thread that runs out raises *abort and records the timeout.
__device__ __forceinline__ bool cl_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                        unsigned int limit, ScanCtl *ctl) {
    for (unsigned int n = 0;; n++) {
        if (cl_try_wait(bar, parity)) return true;
        if ((n & 15u) == 15u && *abort) return false;
        if (n >= limit) {
            *abort = 1;
            atomicExch(&ctl->timeout, 1u);
            return false;
        }
    }
}

}  // namespace

// Sub-tile geometry: TT = 8 P M timesteps per CTA (P = 32 / D lane groups of a warp, each owning
// a run of M timesteps of one channel), E = TT D elements; a cluster tile is CL sub-tiles.
// Shared memory per slot: a and b (E values of S each) and s (E floats), each 16-byte rounded.
// Iteration `it` of every role uses slot it % NS and mbarrier phase it / NS; the publishers take
// the iterations of one parity each and the walkers those of one residue mod 4, so a role always
// finds the phase it waits for at most one completion ahead.
template <typename S, int NS>
__global__ void __launch_bounds__(kThreads, 1)
scan_diag_cluster_kernel(int T, int D, int M, int LAG, const S *__restrict__ a, const S *__restrict__ b,
                         float *__restrict__ s, const float *__restrict__ s_reset, unsigned int *flags,
                         float *__restrict__ gagg, float *__restrict__ gincl, ScanCtl *ctl,
                         EvalStats *stats, const int *skip, unsigned int spin_limit) {
    static_assert(NS % kWalkers == 0 && NS % kPublishers == 0 && NS <= 8, "slots per role");
    if (skip && *(volatile const int *)skip) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar_full[NS], bar_tick[NS], bar_cagg[NS], bar_carry[NS],
        bar_empty[NS], bar_agg[NS];
    __shared__ int slot_tile[NS];
    __shared__ float2 xpre[NS][kCompute];       // per lane: exclusive prefix map of its run in the sub-tile
    __shared__ float carry_all[NS][kMaxCl][32];  // rank 0: the carry into each rank's sub-tile
    __shared__ float2 cagg[NS][kMaxCl][32];      // rank 0: the CTA aggregates of the cluster tile
    __shared__ float2 wagg[2][8][32];            // warp aggregates (double-buffered across tiles)
    __shared__ unsigned int s_epoch;
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t rank = cl_rank(), CL = cl_size();
    const int P = 32 / D, L = P * D;
    const int TT = 8 * P * M;
    const long long CT = (long long)CL * TT;  // timesteps per cluster tile
    const unsigned int ntiles = (unsigned int)((T + CT - 1) / CT);
    const size_t E = (size_t)TT * D;
    const size_t ab_region = (E * sizeof(S) + 15) & ~(size_t)15;
    const size_t s_region = (E * sizeof(float) + 15) & ~(size_t)15;
    const size_t slot_bytes = 2 * ab_region + s_region;
    auto sb = [](const void *p) { return tc::smem_u32(p); };

    if (tid == 0) {
        for (int i = 0; i < NS; i++) {
            tc::mbar_init(sb(&bar_full[i]), 1);
            tc::mbar_init(sb(&bar_tick[i]), 1);
            tc::mbar_init(sb(&bar_cagg[i]), CL);
            tc::mbar_init(sb(&bar_carry[i]), 1);
            tc::mbar_init(sb(&bar_empty[i]), 8);
            tc::mbar_init(sb(&bar_agg[i]), 1);
        }
        tc::fence_barrier_init();
        s_epoch = *(volatile unsigned int *)&ctl->epoch;
        s_abort = 0;
    }
    __syncthreads();
    cl_sync();  // every CTA's barriers are initialised before any remote arrival
    const unsigned int epoch = s_epoch;
    volatile int *abort = &s_abort;
    float dmax = 0.f;
    unsigned int resets = 0;
    // every lane waits (each acquires what the phase publishes); the warp agrees on the outcome
    auto warp_wait = [&](uint32_t bar, uint32_t parity) {
        return __all_sync(0xffffffffu, cl_wait(bar, parity, abort, spin_limit, ctl));
    };
    // the composed aggregate of the cluster tile in slot `slot` (ranks in order), channel `lane`
    auto cluster_agg = [&](int slot, float &TA, float &TB) {
        TA = 1.f;
        TB = 0.f;
        if (lane < D)
            for (uint32_t q = 0; q < CL; q++) {
                const float2 g = cagg[slot][q][lane];
                TB = g.x * TB + g.y;
                TA = g.x * TA;
            }
    };

    if (w == kProducerWarp) {
        // ------------------------------ producer ------------------------------
        int issued = 0;
        for (int it = 0;; it++) {
            const int slot = it % NS;
            const uint32_t ph = (uint32_t)(it / NS) & 1u;
            if (it >= NS && !warp_wait(sb(&bar_empty[slot]), ph ^ 1u)) break;
            if (rank == 0) {  // the ticket goes to every rank, one lane per rank
                unsigned int t = 0;
                if (lane == 0) t = atomicAdd(&ctl->ticket, 1u);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (lane < (int)CL) {
                    cl_st_u32(cl_map(sb(&slot_tile[slot]), lane), t);
                    cl_arrive(cl_map(sb(&bar_tick[slot]), lane));
                }
            }
            if (!warp_wait(sb(&bar_tick[slot]), ph)) break;
            const unsigned int t = (unsigned int)slot_tile[slot];
            if (t >= ntiles) {
                if (lane == 0) {
                    tc::mbar_arrive(sb(&bar_full[slot]));  // releases the compute warps
                    // the publishers and walkers waiting at the next iterations learn the end too
                    if (rank == 0)
                        for (int it2 = it + 1; it2 < it + kWalkers; it2++) {
                            const int slot2 = it2 % NS;
                            const uint32_t ph2 = (uint32_t)(it2 / NS) & 1u;
                            if (it2 >= NS && !cl_wait(sb(&bar_empty[slot2]), ph2 ^ 1u, abort, spin_limit, ctl))
                                break;
                            slot_tile[slot2] = (int)ntiles;
                            tc::mbar_arrive(sb(&bar_tick[slot2]));
                        }
                }
                break;
            }
            if (lane == 0) {
                const long long t0 = (long long)t * CT + (long long)rank * TT;
                const long long tv = min((long long)TT, max(0ll, (long long)T - t0));
                const size_t base = (size_t)max(0ll, t0) * D;
                const size_t Ev = (size_t)tv * D;
                const uint32_t ab_bytes = (uint32_t)((Ev * sizeof(S)) & ~(size_t)15);
                const uint32_t s_bytes = (uint32_t)((Ev * sizeof(float)) & ~(size_t)15);
                unsigned char *buf = smem_raw + (size_t)slot * slot_bytes;
                tc::fence_async_smem();
                tc::mbar_arrive_expect_tx(sb(&bar_full[slot]), 2 * ab_bytes + s_bytes);
                if (ab_bytes) {
                    tc::bulk_g2s(sb(buf), a + base, ab_bytes, sb(&bar_full[slot]));
                    tc::bulk_g2s(sb(buf + ab_region), b + base, ab_bytes, sb(&bar_full[slot]));
                }
                if (s_bytes) tc::bulk_g2s(sb(buf + 2 * ab_region), s + base, s_bytes, sb(&bar_full[slot]));
            }
            issued = it + 1;
        }
        // after an abort: let the copies that were issued land before the block exits
        if (lane == 0 && *abort)
            for (int it = max(0, issued - NS); it < issued; it++)
                tc::mbar_wait_drain(sb(&bar_full[it % NS]), (uint32_t)(it / NS) & 1u, 1u << 20);
    } else if (w >= kPublisherWarp && w < kPublisherWarp + kPublishers) {
        // ------------------------------ publishers (rank 0) ------------------------------
        // the cluster tile's aggregate, published for the look-backs of later tiles (tile 0: its
        // inclusive value)
        if (rank == 0)
            for (int it = w - kPublisherWarp;; it += kPublishers) {
                const int slot = it % NS;
                const uint32_t ph = (uint32_t)(it / NS) & 1u;
                if (!warp_wait(sb(&bar_tick[slot]), ph)) break;
                const unsigned int t = (unsigned int)slot_tile[slot];
                if (t >= ntiles) break;
                if (!warp_wait(sb(&bar_cagg[slot]), ph)) break;
                float TA, TB;
                cluster_agg(slot, TA, TB);
                if (lane < D) {
                    if (t == 0) {
                        gincl[lane] = TB;
                    } else {
                        gagg[((size_t)t * 2) * D + lane] = TA;
                        gagg[((size_t)t * 2 + 1) * D + lane] = TB;
                    }
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) {
                    st_release(flags + t, make_flag(epoch, t == 0 ? kFlagIncl : kFlagAgg));
                    tc::mbar_arrive(sb(&bar_agg[slot]));
                }
            }
    } else if (w >= kWalkerWarp) {
        // ------------------------------ walkers (rank 0) ------------------------------
        if (rank == 0)
            for (int it = w - kWalkerWarp;; it += kWalkers) {
                const int slot = it % NS;
                const uint32_t ph = (uint32_t)(it / NS) & 1u;
                if (!warp_wait(sb(&bar_tick[slot]), ph)) break;
                const unsigned int t = (unsigned int)slot_tile[slot];
                if (t >= ntiles) break;
                if (!warp_wait(sb(&bar_cagg[slot]), ph)) break;
                float TA, TB;
                cluster_agg(slot, TA, TB);
                float c = 0.f;  // carry into the cluster tile, channel `lane`
                if (t > 0) {
                    int jend = (int)t - 1;
                    float GA = 1.f, GB = 0.f;  // composition of the walked predecessors
                    for (;;) {
                        const int j = jend - lane;
                        const unsigned int st = j >= 0 ? wait_flag(flags, j, epoch, spin_limit, ctl) : kFlagIncl;
                        const unsigned int stop = __ballot_sync(0xffffffffu, j < 0 || st != kFlagAgg);
                        const int cnt = stop ? __ffs(stop) - 1 : 32;  // aggregates before the stop
                        const unsigned int stl = __shfl_sync(0xffffffffu, st, stop ? cnt : 0);
                        const int j0 = jend - cnt;
                        if (lane < D) {
                            float ga[32], gb[32];
#pragma unroll
                            for (int i = 0; i < 32; i++) {
                                const bool on = i < cnt;
                                ga[i] = on ? __ldcg(gagg + ((size_t)(jend - i) * 2) * D + lane) : 1.f;
                                gb[i] = on ? __ldcg(gagg + ((size_t)(jend - i) * 2 + 1) * D + lane) : 0.f;
                            }
                            float iv = 0.f;
                            if (stop && j0 >= 0 && stl == kFlagIncl) iv = __ldcg(gincl + (size_t)j0 * D + lane);
#pragma unroll
                            for (int i = 0; i < 32; i++) {  // G <- G o F_i, nearest first
                                GB = GA * gb[i] + GB;
                                GA = GA * ga[i];
                            }
                            if (stop) c = GA * iv + GB;
                        }
                        if (stop) break;
                        jend -= 32;
                    }
                }
                // the carries into the ranks' sub-tiles stay here; each rank reads its own
                if (lane < D) {
                    float cr = c;
                    for (uint32_t q = 0; q < CL; q++) {
                        carry_all[slot][q][lane] = cr;
                        const float2 g = cagg[slot][q][lane];
                        cr = g.x * cr + g.y;
                    }
                }
                // the published aggregate precedes the inclusive value (its flag must not overwrite
                // the inclusive one) and the slot's next use (its barrier phase)
                const bool okp = warp_wait(sb(&bar_agg[slot]), ph);
                cl_fence();
                __syncwarp();
                if (lane < (int)CL) cl_arrive(cl_map(sb(&bar_carry[slot]), lane));
                if (!okp) break;
                if (t > 0) {
                    if (lane < D) gincl[(size_t)t * D + lane] = TA * c + TB;
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) st_release(flags + t, make_flag(epoch, kFlagIncl));
                }
            }
    } else {
        // ------------------------------ compute warps ------------------------------
        const bool lane_on = lane < L;
        const int d = lane_on ? lane % D : 0;
        const int q = lane_on ? lane / D : 0;
        const int last_lane = (P - 1) * D + d;
        const int tg = (w * P + q) * M;  // first local timestep of this lane group's run
        int tiles_ring[8] = {};          // tile of each slot
        auto pass2 = [&](int j) {
            const int slot = j % NS;
            const uint32_t ph = (uint32_t)(j / NS) & 1u;
            const bool ok = warp_wait(sb(&bar_carry[slot]), ph);
            const unsigned int t = (unsigned int)tiles_ring[slot];
            const long long t0 = (long long)t * CT + (long long)rank * TT;
            const int TTv = (int)min((long long)TT, max(0ll, (long long)T - t0));
            const int mv = lane_on ? max(0, min(M, TTv - tg)) : 0;
            unsigned char *buf = smem_raw + (size_t)slot * slot_bytes;
            const S *sa = reinterpret_cast<const S *>(buf);
            const S *sbv = reinterpret_cast<const S *>(buf + ab_region);
            const float *ss = reinterpret_cast<const float *>(buf + 2 * ab_region);
            if (ok && mv > 0) {
                const float2 x = xpre[slot][tid];
                const float cin = cl_ld_f32(cl_map(sb(&carry_all[slot][rank][d]), 0));
                float delta = x.x * cin + x.y;
                const size_t base = (size_t)t0 * D;
#pragma unroll 4
                for (int i = 0; i < mv; i++) {
                    const int e = (tg + i) * D + d;
                    delta = load_as<S, float>(sa + e) * delta + load_as<S, float>(sbv + e);
                    float sn = ss[e] + delta;
                    if (!finite(sn)) {
                        sn = s_reset ? s_reset[d] : 0.f;
                        resets++;
                    } else {
                        dmax = fmaxf(dmax, fabsf(delta));
                    }
                    __stcs(s + base + e, sn);
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(sb(&bar_empty[slot]));
        };
        int it = 0;
        for (;; it++) {
            const int slot = it % NS;
            const uint32_t ph = (uint32_t)(it / NS) & 1u;
            // the compute warps leave together (they share named barriers): the AND of every
            // warp's wait decides
            bool okw = warp_wait(sb(&bar_full[slot]), ph);
            okw = tc::named_bar_and(1, kCompute, okw && !*abort);
            if (!okw) break;
            const unsigned int t = (unsigned int)slot_tile[slot];
            if (t >= ntiles) break;
            tiles_ring[slot] = (int)t;
            const long long t0 = (long long)t * CT + (long long)rank * TT;
            const int TTv = (int)min((long long)TT, max(0ll, (long long)T - t0));
            const int Ev = TTv * D;
            unsigned char *buf = smem_raw + (size_t)slot * slot_bytes;
            S *sa = reinterpret_cast<S *>(buf);
            S *sbv = reinterpret_cast<S *>(buf + ab_region);
            float *ss = reinterpret_cast<float *>(buf + 2 * ab_region);
            const int ab_done = (int)((((size_t)Ev * sizeof(S)) & ~(size_t)15) / sizeof(S));
            const int s_done = (int)((((size_t)Ev * sizeof(float)) & ~(size_t)15) / sizeof(float));
            if (ab_done < Ev || s_done < Ev) {  // uniform: the sub-16-byte tail of the chain
                const size_t base = (size_t)t0 * D;
                for (int e = ab_done + tid; e < Ev; e += kCompute) {
                    sa[e] = a[base + e];
                    sbv[e] = b[base + e];
                }
                for (int e = s_done + tid; e < Ev; e += kCompute) ss[e] = s[base + e];
                compute_bar();
            }
            const int mv = lane_on ? max(0, min(M, TTv - tg)) : 0;
            // pass 1: the run's composed map
            float GA = 1.f, GB = 0.f;
#pragma unroll 4
            for (int i = 0; i < mv; i++) {
                const int e = (tg + i) * D + d;
                const float ra = load_as<S, float>(sa + e);
                GB = ra * GB + load_as<S, float>(sbv + e);
                GA = ra * GA;
            }
            // inclusive scan over the P runs of the warp (channel-segmented)
            float IA = GA, IB = GB;
            for (int off = D; off < L; off <<= 1) {
                const float pa = __shfl_up_sync(0xffffffffu, IA, off);
                const float pb = __shfl_up_sync(0xffffffffu, IB, off);
                if (lane_on && lane >= off) {
                    IB = IA * pb + IB;
                    IA = IA * pa;
                }
            }
            // exclusive prefix of the run within the warp (identity for the first group)
            float XA = __shfl_up_sync(0xffffffffu, IA, D), XB = __shfl_up_sync(0xffffffffu, IB, D);
            if (lane < D) {
                XA = 1.f;
                XB = 0.f;
            }
            {
                const float ea = __shfl_sync(0xffffffffu, IA, last_lane);
                const float eb = __shfl_sync(0xffffffffu, IB, last_lane);
                if (lane < D) wagg[it & 1][w][lane] = make_float2(ea, eb);
            }
            compute_bar();
            // prefix over the earlier warps, then the run's exclusive prefix map in the sub-tile
            {
                float PA = 1.f, PB = 0.f;
                for (int k = 0; k < w; k++) {
                    const float2 g = wagg[it & 1][k][d];
                    PB = g.x * PB + g.y;
                    PA = g.x * PA;
                }
                xpre[slot][tid] = make_float2(XA * PA, XA * PB + XB);
            }
            if (w == 0) {  // the CTA aggregate goes to rank 0
                if (lane < D) {
                    float CA = 1.f, CB = 0.f;
                    for (int k = 0; k < 8; k++) {
                        const float2 g = wagg[it & 1][k][lane];
                        CB = g.x * CB + g.y;
                        CA = g.x * CA;
                    }
                    const uint32_t dst = cl_map(sb(&cagg[slot][rank][lane]), 0);
                    cl_st_f32(dst, CA);
                    cl_st_f32(dst + 4, CB);
                    cl_fence();
                }
                __syncwarp();
                if (lane == 0) cl_arrive(cl_map(sb(&bar_cagg[slot]), 0));
            }
            if (it >= LAG) pass2(it - LAG);
        }
        // drain: pass 2 of the tiles still waiting for their carries (after an abort the waits
        // give up at once and only release the slots)
        for (int j = max(0, it - LAG); j < it; j++) pass2(j);
    }
    __syncthreads();
    if (stats) block_stats(stats, (double)dmax, resets);
    cl_sync();  // no CTA leaves while another may still address its shared memory
    exit_persistent(ctl);
}

// ---- host side ---------------------------------------------------------------------------------

namespace {

// Cluster size: PMCMC_SCAN_CLUSTER = 2, 4 or 8 (read at every call; default 8).
int cluster_size() {
    const char *e = getenv("PMCMC_SCAN_CLUSTER");
    const int v = e ? atoi(e) : 8;
    return (v == 2 || v == 4 || v == 8) ? v : 8;
}

// Shared memory of the kernel besides the slots (the static arrays), rounded up.
template <int NS>
constexpr size_t cluster_static_smem() {
    return (size_t)NS * (6 * 8 + 4 + kCompute * 8 + kMaxCl * 32 * 4 + kMaxCl * 32 * 8) + 2 * 8 * 32 * 8 + 2048;
}

// Run length M: NS slots of a, b and s within the dynamic shared memory left beside the static
// arrays; M - 1 a multiple of 32 / gcd(D, 32) (the P runs of a warp then start in distinct
// banks) unless that would halve the run.
template <int NS>
int cluster_run(int D, int sbytes) {
    const int P = 32 / D;
    const size_t dyn = 227 * 1024 - cluster_static_smem<NS>();
    const size_t per_slot = dyn / NS - 48;
    const int cap = std::max(1, (int)(per_slot / ((size_t)8 * P * D * (2 * sbytes + 4))));
    if (P == 1) return cap;
    const int c = 32 / std::gcd(D, 32);
    const int m = (cap - 1) / c * c + 1;
    return 2 * m >= cap ? m : cap;
}

template <typename S>
size_t cluster_slot_bytes(int M, int D) {
    const size_t E = (size_t)8 * (32 / D) * M * D;
    return 2 * ((E * sizeof(S) + 15) & ~(size_t)15) + ((E * 4 + 15) & ~(size_t)15);
}

template <typename S, int NS>
cudaError_t run_scan_cluster(int T, int D, const void *a, const void *b, void *s, const void *s_reset,
                             const ScanWork &w, EvalStats *stats, const int *skip, unsigned int spin,
                             cudaStream_t st) {
    const int CL = cluster_size();
    const int M = cluster_run<NS>(D, (int)sizeof(S));
    const long long CT = (long long)CL * 8 * (32 / D) * M;
    const int ntiles = (int)((T + CT - 1) / CT);
    if (ntiles > w.max_tiles) return cudaErrorInvalidValue;
    const char *le = getenv("PMCMC_SCAN_LAG");
    int lag = le ? atoi(le) : 2;
    lag = std::max(1, std::min(lag, NS - 2));
    const size_t smem = (size_t)NS * cluster_slot_bytes<S>(M, D);
    auto k = scan_diag_cluster_kernel<S, NS>;
    cudaError_t e = ensure_dyn_smem(k, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // persistent: at most the clusters that can be resident at once (cached per configuration)
    static int cached_key[16][3], cached_val[16], ncached = 0;
    int nclusters = 0;
    for (int i = 0; i < ncached; i++)
        if (cached_key[i][0] == CL && cached_key[i][1] == (int)smem && cached_key[i][2] == NS)
            nclusters = cached_val[i];
    if (nclusters == 0) {
        cfg.gridDim = dim3(CL * 152);
        if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            return cudaErrorInvalidConfiguration;
        }
        if (ncached < 16) {
            cached_key[ncached][0] = CL;
            cached_key[ncached][1] = (int)smem;
            cached_key[ncached][2] = NS;
            cached_val[ncached++] = nclusters;
        }
    }
    cfg.gridDim = dim3(CL * std::min(ntiles, nclusters));
    return cudaLaunchKernelEx(&cfg, k, T, D, M, lag, (const S *)a, (const S *)b, (float *)s,
                              (const float *)s_reset, w.flags, (float *)w.agg, (float *)w.incl, w.ctl,
                              stats, skip, spin);
}

}  // namespace

// Timesteps per cluster tile for (D, element size): sizes the look-back workspace.
int diag_scan_tile_cluster(int D, int sbytes) {
    const char *e = getenv("PMCMC_SCAN_SLOTS");
    const int M = (e && atoi(e) == 8) ? cluster_run<8>(D, sbytes) : cluster_run<4>(D, sbytes);
    return cluster_size() * 8 * (32 / D) * M;
}

// Diagonal scan of FP32 iterates on thread-block clusters (D <= 32; a and b FP32 or bfloat16;
// a, b and s 16-byte aligned).  PMCMC_SCAN_SLOTS = 8 selects eight sub-tile slots per CTA
// (default four).
cudaError_t launch_scan_diag_cluster(int storage, int T, int D, const void *a, const void *b, void *s,
                                     const void *s_reset, const ScanWork &w, EvalStats *stats,
                                     const int *skip, unsigned int spin_limit, cudaStream_t st) {
    const char *e = getenv("PMCMC_SCAN_SLOTS");
    const bool eight = e && atoi(e) == 8;
    if (storage == 1)
        return eight ? run_scan_cluster<__nv_bfloat16, 8>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st)
                     : run_scan_cluster<__nv_bfloat16, 4>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    return eight ? run_scan_cluster<float, 8>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st)
                 : run_scan_cluster<float, 4>(T, D, a, b, s, s_reset, w, stats, skip, spin_limit, st);
}

}  // namespace pm
