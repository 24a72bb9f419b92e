// Dense scan (DEER, Eq. 3) with the D x D compositions on the tensor cores, D <= 32:
//   delta_t = J_t delta_{t-1} + b_t,   s_t <- s_t + delta_t,
// the variant of the precision F32_SCAN_BF16 (the Jacobian compositions in bfloat16 with FP32
// accumulation; the Newton loop, whose residual is formed in FP32, refines the solve).
//
// A CTA takes a tile of four chunks of C timesteps.  Phase A builds each chunk's transfer
// product P = J_{C-1} ... J_0 on the tensor cores: at step i the four chunks' products
// P_i = J_i P_{i-1} are one tcgen05.mma of kind::f16 with M = 128 (four chunks of 32 rows),
// N = 32 and K = 128 against a block-diagonal A operand (the four J_i on its diagonal: three
// quarters of the products are zeros, the price of putting 32 x 32 products on an M = 128
// tile) and the four P_{i-1} stacked along K as the B operand.  The accumulator goes back from
// TMEM through registers to the B operand of the next step (bfloat16, transposed write); the
// next step's J rows are converted into the other A buffer while the MMA runs.  The chunk's
// local vector b (zero carry) runs alongside in FP32 on the CUDA cores.
// Phase B composes the four chunk maps into the tile aggregate (FP32) and resolves the carry by
// a decoupled look-back over tiles (nearest inclusive predecessor, aggregates in between applied
// as matrix-vector products).  Phase C re-runs each chunk's recursion in FP32 from its carry and
// updates s, so only the carry passes through the bfloat16 products.
// Every wait is bounded: a wait that runs out sets the launch's timeout word and the CTA
// finishes without further work (in-flight MMAs drained, TMEM freed).
#include "common.cuh"
#include "internal.h"
#include "lookback.cuh"
#include "tc.cuh"

namespace pm {
namespace {

using namespace tc;

constexpr int kP = 32;                 // padded state dimension
constexpr int kNChunk = 4;             // chunks per tile (the four 32-row blocks of M = 128)
constexpr int kEpi = 4;                // one warp per chunk
constexpr int kThreads = (kEpi + 1) * 32;  // + the MMA-issuer warp
constexpr int kIss = kEpi;
constexpr int kARegion = 128 * 128;    // bytes of one 64-column K region of the 128 x 128 A operand
constexpr int kABuf = 2 * kARegion;    // K = 128 bfloat16 = two regions
constexpr int kBRegion = 32 * 128;     // one K region of the 32 x 128 B operand
constexpr int oA = 0;                  // two A buffers
constexpr int oB = 2 * kABuf;          // B operand (two regions)
constexpr int oP = oB + 2 * kBRegion;  // FP32 chunk products [4][32][33] after phase A
constexpr int kPStride = 33;
constexpr int oBv = oP + kNChunk * 32 * kPStride * 4;  // b vectors [2][4][32]
constexpr int oTA = oBv + 2 * kNChunk * 32 * 4;        // tile aggregate A [32][33] (FP32)
constexpr int oTmp = oTA + 32 * kPStride * 4;          // product scratch [32][33]
constexpr int oVec = oTmp + 32 * kPStride * 4;         // vectors [8][32]
constexpr int oBar = (oVec + 8 * 32 * 4 + 7) & ~7;
constexpr int kNBar = 5;                               // A ready (x2), MMA done, look-back copies (x2)
constexpr int oMisc = oBar + 8 * kNBar;
constexpr int kSmemUsed = oMisc + 32;
constexpr int kSmemBytes = kSmemUsed + 1024;
constexpr unsigned int kDrain = 1u << 20;

// instruction descriptor of kind::f16 with bfloat16 A and B, FP32 accumulator, both K-major
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_bf16(128, 32);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// byte offset of bfloat16 element (row, k) in a K-major 128-byte-swizzled operand whose K is
// split into 64-column regions of `region_bytes` each
__device__ __forceinline__ uint32_t swz_bf16(uint32_t row, uint32_t k, uint32_t region_bytes) {
    const uint32_t kr = k & 63u;
    return (k >> 6) * region_bytes + (row >> 3) * 1024u + (row & 7u) * 128u +
           ((((kr >> 3) ^ (row & 7u)) & 7u) << 4) + (kr & 7u) * 2u;
}

__device__ __forceinline__ void st_bf16(unsigned char *base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// elements k and k + 1 (k even) of one operand row: adjacent in the swizzled layout
__device__ __forceinline__ void st_bf16x2(unsigned char *base, uint32_t off, float v0, float v1) {
    *reinterpret_cast<__nv_bfloat162 *>(base + off) = __floats2bfloat162_rn(v0, v1);
}

// Warp-uniform bounded wait (every lane polls; every lane takes the same branch afterwards).
__device__ __forceinline__ bool warp_all_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                              unsigned int limit) {
    const bool ok = mbar_wait(bar, parity, abort, limit);
    return __all_sync(0xffffffffu, ok);
}

// SA, SB: storage of the Jacobians and of the right-hand sides (float or bfloat16)
template <typename SA, typename SB>
__global__ void __launch_bounds__(kThreads, 1)
scan_dense_tc_kernel(int T, int D, int C, const SA *__restrict__ a, const SB *__restrict__ b,
                     float *__restrict__ s, const float *__restrict__ s_reset, unsigned int *flags,
                     float *__restrict__ gagg, float *__restrict__ gincl, ScanCtl *ctl,
                     EvalStats *stats, const int *skip, unsigned int spin_limit) {
    if (skip && *(volatile const int *)skip) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const uint32_t sb = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int DD = D * D;
    const size_t AGG = (size_t)dense_agg_stride(D);  // 16-byte aligned aggregates
    const unsigned int limit = spin_limit ? spin_limit : kDefaultSpinLimit;
    volatile int *abort_f = reinterpret_cast<volatile int *>(sm + oMisc + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + oMisc);
    unsigned int *tile_slot = reinterpret_cast<unsigned int *>(sm + oMisc + 8);
    auto bar = [&](int i) -> uint32_t { return sb + oBar + 8u * (uint32_t)i; };
    const unsigned int ntiles = (unsigned int)ceil_div(T, kNChunk * C);

    // zero both A buffers (off-diagonal blocks stay zero), barriers, ticket
    for (int e = tid; e < (2 * kABuf) / 16; e += kThreads)
        reinterpret_cast<uint4 *>(sm + oA)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(bar(0), kEpi);
        mbar_init(bar(1), kEpi);
        mbar_init(bar(2), 1);
        mbar_init(bar(3), 1);
        mbar_init(bar(4), 1);
        *abort_f = 0;
        tile_slot[0] = atomicAdd(&ctl->ticket, 1u);
        tile_slot[1] = *(volatile unsigned int *)&ctl->epoch;
        fence_barrier_init();
    }
    if (warp == kIss) {
        tmem_alloc(smem_u32(tmem_slot), 32);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tmem_slot;
    const int tile = (int)tile_slot[0];
    const unsigned int epoch = tile_slot[1];
    const int t0 = tile * kNChunk * C;

    float *Pm = reinterpret_cast<float *>(sm + oP);
    float *bv = reinterpret_cast<float *>(sm + oBv);
    bool ok = true;

    // ---------------- phase A: chunk products on the tensor cores ----------------
    int ncommit = 0;  // MMA steps issued (issuer lane)
    if (warp == kIss) {
        if (lane == 0) {
            for (int i = 1; i < C && ok; i++) {
                if (!(ok = mbar_wait(bar(i & 1), (uint32_t)((i - 1) >> 1) & 1u, abort_f, limit))) break;
                tc_fence_after();
                const uint32_t ab = sb + oA + (uint32_t)(i & 1) * kABuf;
#pragma unroll
                for (int kk = 0; kk < 8; kk++) {
                    const uint32_t reg = (uint32_t)(kk >> 2), kin = (uint32_t)(kk & 3) * 32u;
                    mma_bf16(tm, sdesc(ab + reg * kARegion + kin), sdesc(sb + oB + reg * kBRegion + kin),
                             kIdesc, kk > 0 ? 1u : 0u);
                }
                mma_commit(bar(2));
                ncommit++;
            }
            // No commit follows the last step's: a further completion of the same barrier could
            // complete the phase after the one the epilogue waits for before it looks, and a
            // parity wait would then miss it.
        }
        __syncwarp();
    } else {
        const int c = warp, r = lane;          // chunk c of the tile, row r of its matrices
        const int tc0 = t0 + c * C;            // first timestep of the chunk
        const uint32_t lrow = tm + ((uint32_t)(32 * c) << 16);
        float jr[kP], jn[kP], jn2[kP];
        // row r of J_t (identity beyond T) and b_t[r] (zero beyond T)
        auto load_row = [&](int t, float (&v)[kP], float &bb) {
            const bool in = t < T;
#pragma unroll
            for (int k = 0; k < kP; k++)
                v[k] = (in && r < D && k < D) ? ldg_as<SA, float>(a + (size_t)t * DD + (size_t)r * D + k)
                                              : ((!in && k == r) ? 1.0f : 0.0f);
            bb = (in && r < D) ? ldg_as<SB, float>(b + (size_t)t * D + r) : 0.0f;
        };
        // step 0: P_0 = J_0, b_0 = b_{t0}; the rows of the next two steps are always in flight
        float bcur, bn = 0.0f, bn2 = 0.0f;
        load_row(tc0, jr, bcur);
        if (C > 1) load_row(tc0 + 1, jn, bn);
        if (C > 2) load_row(tc0 + 2, jn2, bn2);
        bv[(0 * kNChunk + c) * 32 + r] = bcur;
#pragma unroll
        for (int n = 0; n < kP; n++) st_bf16(sm + oB, swz_bf16((uint32_t)n, (uint32_t)(32 * c + r), kBRegion), jr[n]);
        for (int i = 1; i < C; i++) {
            float acc = bn;
#pragma unroll
            for (int k = 0; k < kP; k++) {
                jr[k] = jn[k];
                jn[k] = jn2[k];
            }
            bn = bn2;
            if (i + 2 < C) load_row(tc0 + i + 2, jn2, bn2);
            __syncwarp();  // b_{i-1} of every row of the chunk is in shared memory
            const float *bp = bv + (((i - 1) & 1) * kNChunk + c) * 32;
#pragma unroll
            for (int k = 0; k < kP; k++) acc = fmaf(jr[k], bp[k], acc);
            bv[((i & 1) * kNChunk + c) * 32 + r] = acc;
            bcur = acc;
            // A operand of step i: row 32 c + r, K columns 32 c .. 32 c + 31
            unsigned char *ab = sm + oA + (i & 1) * kABuf;
#pragma unroll
            for (int k = 0; k < kP; k += 2)
                st_bf16x2(ab, swz_bf16((uint32_t)(32 * c + r), (uint32_t)(32 * c + k), kARegion), jr[k], jr[k + 1]);
            if (i >= 2) {  // B operand: P_{i-1}, the result of step i - 1
                if (!(ok = warp_all_wait(bar(2), (uint32_t)(i - 2) & 1u, abort_f, limit))) break;
                tc_fence_after();
                float pr[kP];
                tmem_ld16(lrow, pr);
                tmem_ld16(lrow + 16u, pr + 16);
                tmem_wait_ld();
#pragma unroll
                for (int n = 0; n < kP; n++) st_bf16(sm + oB, swz_bf16((uint32_t)n, (uint32_t)(32 * c + r), kBRegion), pr[n]);
            }
            fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(i & 1));
        }
        // the chunk product (FP32) and b: P = P_{C-1}
        float pr[kP];
        if (ok && C >= 2) {
            ok = warp_all_wait(bar(2), (uint32_t)(C - 2) & 1u, abort_f, limit);
            tc_fence_after();
            if (ok) {
                tmem_ld16(lrow, pr);
                tmem_ld16(lrow + 16u, pr + 16);
                tmem_wait_ld();
            }
        } else {
#pragma unroll
            for (int n = 0; n < kP; n++) pr[n] = jr[n];
        }
#pragma unroll
        for (int n = 0; n < kP; n++) Pm[(c * 32 + r) * kPStride + n] = ok ? pr[n] : 0.0f;
        bv[(0 * kNChunk + c) * 32 + r] = bcur;  // chunk vector, slot 0
    }
    // drain: the last step's completion (also when the epilogue gave up early)
    if (warp == kIss && lane == 0 && ncommit > 0) mbar_wait_drain(bar(2), (uint32_t)(ncommit - 1) & 1u, kDrain);
    tc_fence_before();
    __syncthreads();
    if (warp == kIss) {
        tc_fence_after();
        tmem_dealloc(tm, 32);
    }
    if (*abort_f && tid == 0) atomicExch(&ctl->timeout, 1u);

    // ---------------- phase B: tile aggregate and the carry by look-back ----------------
    // tile map = M3 o M2 o M1 o M0 (FP32 on the CUDA cores): TA = P3 P2 P1 P0, tb by matvecs
    float *TA = reinterpret_cast<float *>(sm + oTA);
    float *tmp = reinterpret_cast<float *>(sm + oTmp);
    float *vec = reinterpret_cast<float *>(sm + oVec);
    for (int e = tid; e < kP * kP; e += kThreads) TA[(e >> 5) * kPStride + (e & 31)] = Pm[(e >> 5) * kPStride + (e & 31)];
    if (tid < kP) vec[tid] = bv[tid];  // chunk 0's b
    __syncthreads();
    for (int c = 1; c < kNChunk; c++) {
        const float *Pc = Pm + c * 32 * kPStride;
        for (int e = tid; e < kP * kP; e += kThreads) {
            const int i = e >> 5, j = e & 31;
            float acc = 0.0f;
            for (int k = 0; k < kP; k++) acc = fmaf(Pc[i * kPStride + k], TA[k * kPStride + j], acc);
            tmp[i * kPStride + j] = acc;
        }
        float nb = 0.0f;
        if (tid < kP) {
            nb = bv[c * 32 + tid];
            for (int k = 0; k < kP; k++) nb = fmaf(Pc[tid * kPStride + k], vec[k], nb);
        }
        __syncthreads();
        for (int e = tid; e < kP * kP; e += kThreads) TA[(e >> 5) * kPStride + (e & 31)] = tmp[(e >> 5) * kPStride + (e & 31)];
        if (tid < kP) vec[tid] = nb;
        __syncthreads();
    }
    // publish (tile 0: inclusive value = its own map applied to zero)
    if (tile == 0) {
        if (tid < D) gincl[tid] = vec[tid];
    } else {
        for (int e = tid; e < DD; e += kThreads) gagg[(size_t)tile * AGG + e] = TA[(e / D) * kPStride + (e % D)];
        if (tid < D) gagg[(size_t)tile * AGG + DD + tid] = vec[tid];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(flags + tile, make_flag(epoch, tile == 0 ? kFlagIncl : kFlagAgg));
    float *carry = vec + 32;  // vec[32..63]: the carry into the tile
    if (tid < kP) carry[tid] = 0.0f;
    __syncthreads();
    if (tile > 0) {
        // the A and B operand buffers are free after phase A: they stage the aggregates, two
        // batches of nb
        constexpr int kStageBytes = 2 * kABuf + 2 * kBRegion;
        const int nb = min(32, kStageBytes / (2 * (int)sizeof(float) * dense_agg_stride(D)));
        lookback_dense<float>(flags, gagg, gincl, tile, D, epoch, limit, ctl,
                              reinterpret_cast<float *>(sm + oA), nb, bar(3), carry);
        if (tid < D) {  // inclusive value of this tile = TA carry + tb
            float acc = vec[tid];
            for (int k = 0; k < D; k++) acc = fmaf(TA[tid * kPStride + k], carry[k], acc);
            gincl[(size_t)tile * D + tid] = acc;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(flags + tile, make_flag(epoch, kFlagIncl));
    }

    // ---------------- phase C: each chunk's recursion in FP32 from its carry ----------------
    // carries into the chunks: c_0 = carry, c_{k+1} = P_k c_k + b_k (warp 0)
    float *cin = vec + 128;  // [4][32]
    if (warp == 0) {
        float cv = carry[lane];
        cin[lane] = cv;
        for (int c = 0; c + 1 < kNChunk; c++) {
            float acc = bv[c * 32 + lane];
            for (int k = 0; k < kP; k++) acc = fmaf(Pm[(c * 32 + lane) * kPStride + k], __shfl_sync(0xffffffffu, cv, k), acc);
            cv = acc;
            cin[(c + 1) * 32 + lane] = cv;
        }
    }
    __syncthreads();
    float dmax = 0.0f;
    unsigned int resets = 0;
    if (warp < kEpi) {
        const int c = warp, r = lane;
        float dl = cin[c * 32 + r];
        const int tb = t0 + c * C, te = min(tb + C, T);
        // row r of J_t, b_t[r] and s_t[r] in registers, loaded two steps ahead (zeros for r >= D)
        float jn[kP], jn2[kP], bn = 0.0f, bn2 = 0.0f, sv = 0.0f, sv2 = 0.0f;
        auto load_c = [&](int t, float (&jv)[kP], float &bb, float &ss) {
#pragma unroll
            for (int k = 0; k < kP; k++)
                jv[k] = (r < D && k < D) ? ldg_as<SA, float>(a + (size_t)t * DD + (size_t)r * D + k) : 0.0f;
            bb = r < D ? ldg_as<SB, float>(b + (size_t)t * D + r) : 0.0f;
            ss = r < D ? s[(size_t)t * D + r] : 0.0f;
        };
        if (tb < te) load_c(tb, jn, bn, sv);
        if (tb + 1 < te) load_c(tb + 1, jn2, bn2, sv2);
        for (int t = tb; t < te; t++) {
            float jc[kP];
#pragma unroll
            for (int k = 0; k < kP; k++) {
                jc[k] = jn[k];
                jn[k] = jn2[k];
            }
            float acc = bn;
            const float scur = sv;
            bn = bn2;
            sv = sv2;
            if (t + 2 < te) load_c(t + 2, jn2, bn2, sv2);
#pragma unroll
            for (int k = 0; k < kP; k++) acc = fmaf(jc[k], __shfl_sync(0xffffffffu, dl, k), acc);
            dl = r < D ? acc : 0.0f;
            if (r < D) {
                const size_t o = (size_t)t * D + r;
                float sn = scur + dl;
                if (!isfinite(sn)) {
                    sn = s_reset ? s_reset[r] : 0.0f;
                    resets++;
                } else {
                    dmax = fmaxf(dmax, fabsf(dl));
                }
                s[o] = sn;
            }
        }
    }
    if (stats && warp < kEpi) {
        const float dm = warp_max(dmax);
        const unsigned int rs = __reduce_add_sync(0xffffffffu, resets);
        if (lane == 0) {
            if (dm > 0.0f) atomic_max_d(&stats->dmax, (double)dm);
            if (rs) atomicAdd(&stats->resets, (unsigned long long)rs);
        }
    }
    // the last tile resets the ticket and advances the epoch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int d = atomicAdd(&ctl->done, 1u);
        if (d == ntiles - 1) {
            ctl->ticket = 0;
            ctl->done = 0;
            ctl->epoch = ctl->epoch + 1u;
            __threadfence();
        }
    }
}

}  // namespace

// chunk length: the tiles of one wave (one CTA per SM, 152 SMs: the occupancy this kernel gets)
// share the timesteps, so the serial chain of each tile is as short as one wave allows; 8 to
// 256 timesteps (beyond 4 x 152 x 256 timesteps the tiles take several waves)
int dense_tc_chunk(int T) { return std::min(256, std::max(8, ceil_div(T, kNChunk * 152))); }

template <typename SA, typename SB>
static cudaError_t run_dense_tc(int T, int D, int C, const void *a, const void *b, void *s,
                                const void *s_reset, const ScanWork &w, EvalStats *stats,
                                const int *skip, unsigned int spin_limit, cudaStream_t st) {
    const int ntiles = ceil_div(T, kNChunk * C);
    if (ntiles > w.max_tiles) return cudaErrorInvalidValue;
    auto k = scan_dense_tc_kernel<SA, SB>;
    cudaError_t e = ensure_dyn_smem(k, kSmemBytes);
    if (e != cudaSuccess) return e;
    k<<<ntiles, kThreads, kSmemBytes, st>>>(T, D, C, (const SA *)a, (const SB *)b, (float *)s,
                                            (const float *)s_reset, w.flags, (float *)w.agg,
                                            (float *)w.incl, w.ctl, stats, skip, spin_limit);
    return cudaGetLastError();
}

cudaError_t launch_scan_dense_tc(bool a_bf16, int T, int D, int C, const void *a, const void *b,
                                 void *s, const void *s_reset, const ScanWork &w, EvalStats *stats,
                                 const int *skip, unsigned int spin_limit, cudaStream_t st) {
    if (D < 1 || D > kP || C < 1) return cudaErrorInvalidValue;
    if (a_bf16)
        return run_dense_tc<__nv_bfloat16, __nv_bfloat16>(T, D, C, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    return run_dense_tc<float, __nv_bfloat16>(T, D, C, a, b, s, s_reset, w, stats, skip, spin_limit, st);
}

}  // namespace pm
