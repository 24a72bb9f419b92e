// Evaluate-and-linearise pass of MALA on Bayesian logistic regression (Section 5.2 target) on
// the fifth-generation tensor cores: tcgen05.mma of kind::tf32 with FP32 accumulators in
// tensor memory (TMEM).  Covers D <= 32, FP32 arithmetic, the exact diagonal of the held-gate
// Jacobian (Section 3.2 with the gate value held) or the zero Jacobian.
//
// Per timestep t a MALA linearisation needs, with x = s_{t-1} and x~ the proposal,
//   z = X x,  g(x) = X^T (y - sigmoid(z)) - x / sp^2,  sum_n [y z - softplus(z)],
//   diag(X^T W X), W = diag(sigmoid'(z))           (pass 1, at x)
//   the same gradient and log-likelihood at x~     (pass 2)
// For a CTA of 128 timesteps the contractions are GEMMs against the shared design matrix:
//   Z = V X^T (128 x N),  G = C X (128 x D),  H = W (X.X) (128 x D),
// computed in chunks of 32 design rows.  Each FP32 operand is split a = a_hi + a_lo into two
// tf32 values and a b is accumulated as (a_hi + a_lo)(b_hi + b_lo) in two MMAs of N = 64 (see
// kIdesc64); the diagonal Hessian H only shapes the Newton step and takes the single product
// a_hi b_hi.
//
// Warp roles (kGroups = 2: 384 threads, one CTA per SM):
//   warps 0-7  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one timestep per lane) and
//              belongs to warpgroup h = w / 4, which owns columns 16h..16h+15 of every chunk and
//              dimensions 16h..16h+15 of the state.  Z -> c = y - sigmoid(z), w = sigmoid'(z)
//              and the log-likelihood terms; c, w are written as tf32 pairs into shared memory
//              as the A operand of G and H.  Each warpgroup forms its dimensions of the
//              proposal, of the residual and of J; the MH log-ratio (FP64) is summed over the
//              warpgroups through shared memory.  (Four warpgroups of 8 columns also compile:
//              they issue 27% more instructions, as each warp repeats the per-chunk waits,
//              accumulator reads and hand-offs, for about the same time.)
//   warps 8-11 control, one per SM sub-partition: warp 8 allocates TMEM and issues the Z
//              products, warp 9 issues the G and H products, lane 0 of warp 10 streams
//              pre-swizzled design chunks with bulk copies (4 stages), warp 11 is idle.
// TMEM: Z in three buffers, G per chunk in two buffers (64 columns each: the B_hi and B_lo
// parts), H accumulated over the chunks.  The tensor core's FP32 accumulation truncates, so
// a sum over all N rows in one accumulator would drift by up to an ulp of |G| per MMA; each
// chunk's G product therefore starts a fresh accumulator and the epilogue adds the 32-row
// partials in registers with round-to-nearest.  Every wait is bounded: a wait that runs out
// raises the CTA's abort flag, the roles finish without further work, in-flight copies and
// MMAs are drained, TMEM is freed and the launch's timeout word is set.
#include <type_traits>

#include "common.cuh"
#include "eval.h"
#include "internal.h"
#include "lookback.cuh"
#include "solve.h"
#include "tc.cuh"

namespace pm {

namespace {

using namespace tc;

constexpr int kM = 128;                        // timesteps per CTA (MMA M; one TMEM lane each)
constexpr int kNB = 32;                        // design rows per chunk
constexpr int kDP = 32;                        // padded feature dimension
constexpr int kStages = 4;                     // chunk images in flight
constexpr int kGroups = 2;                     // epilogue warpgroups
constexpr int kCols = kDP / kGroups;           // columns / dimensions per warpgroup: 8
constexpr int kEpiWarps = 4 * kGroups;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = kEpiThreads + 128;    // + four control warps, one per SM sub-partition
// control warps (lane 0 of each): the Z-product issuer, the G/H-product issuer, the bulk-copy
// producer, and one spare; warp w runs on sub-partition w % 4, so each sub-partition hosts four
// epilogue warps and one control warp
constexpr int kIssZ = kEpiWarps, kIssG = kEpiWarps + 1, kCopyWarp = kEpiWarps + 2;
constexpr int kMmaWarp = kIssZ;                // allocates / frees TMEM
constexpr int kCopyLane = 0;
constexpr int kOp = kNB * kDP * 4;             // one 32 x 32 operand block: 4096 bytes
constexpr int kImg = 5 * kOp + kNB * 4;        // chunk image: X hi, X lo, X^T hi, X^T lo, (X.X)^T hi, y
constexpr int kStageStride = 21504;            // 1024-aligned stage slot
constexpr int kRowOp = kM * kDP * 4;           // a 128 x 32 A operand: 16384 bytes
constexpr uint32_t kIdesc = idesc_tf32(kM, 32);
// The hi and lo blocks of each design operand are adjacent in the chunk image, i.e. one 64-row
// operand [B_hi; B_lo]: a single N=64 MMA multiplies A by both (an MMA of N <= 64 costs about
// the same as N = 32), so a K-step of Z or G takes two MMAs (A_hi and A_lo) instead of three.
// Columns 0-31 of the 64-column result hold A B_hi, columns 32-63 hold A B_lo.
constexpr uint32_t kIdesc64 = idesc_tf32(kM, 64);
constexpr uint32_t kTmemCols = 512;
constexpr unsigned int kDrainLimit = 1u << 20;  // polls of up to ~2 us each

// shared-memory map, offsets from a 1024-aligned base
constexpr int oVhi = 0, oVlo = kRowOp;         // A operand of Z: the states (x, then x~)
constexpr int oCW = 2 * kRowOp;                // 2 buffers of (C hi, C lo, W hi)
constexpr int kCWStride = 3 * kRowOp;
constexpr int oStage = oCW + 2 * kCWStride;
constexpr int oBar = oStage + kStages * kStageStride;
constexpr int kZbuf = 3;                       // Z buffers in TMEM (GEMM1 runs 3 chunks ahead)
constexpr uint32_t kColZ = 0;                  // Z: 3 buffers of 64 columns (hi part, lo part)
constexpr uint32_t kColG = 64 * kZbuf;         // G: 2 buffers of 64 columns (fresh per chunk)
constexpr uint32_t kColH = kColG + 128;        // H: 32 columns
// cfull has four barriers (chunk k uses k % 4) so that no waiter can see a barrier two phases
// ahead: the Z issuer waits on chunks up to four behind the epilogue's newest
constexpr int bFull = 0, bEmpty = kStages, bZfull = 2 * kStages, bCfull = bZfull + kZbuf,
              bCempty = bCfull + 4, bGdone = bCempty + 2, bVready = bGdone + 1, bFin = bVready + 1,
              kNumBars = bFin + 1;
constexpr int oMisc = oBar + 8 * kNumBars;     // tmem address, abort flag
constexpr int oPart = oMisc + 16;              // double [4][128]: per-warpgroup log-ratio parts
constexpr int oAcc = oPart + kGroups * kM * 8; // int [128]: decisions
constexpr int oRed = oAcc + kM * 4;            // double [16][4]: per-warp statistics
constexpr int oLogu = oRed + kEpiWarps * 4 * 8; // double [128]: log u of each timestep
// fused Newton update: per-warp scan totals [16 warps][8 channels][A, B], the carries into the
// four warps of a warpgroup [4][32] (A and B), the 16 segment compositions of the earlier tiles'
// aggregates, the tile carry [32]
constexpr int oFw = oLogu + kM * 8;
constexpr int oFpre = oFw + kEpiWarps * kCols * 2 * 4;
constexpr int oFseg = oFpre + 4 * 32 * 2 * 4;      // [16][32] (A, B): segment compositions
constexpr int oFcar = oFseg + kEpiWarps * 32 * 2 * 4;
constexpr int kSmemUsed = oFcar + 32 * 4;
constexpr int kSmemBytes = kSmemUsed + 1024;   // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(oStage % 1024 == 0 && kStageStride % 1024 == 0 && oCW % 1024 == 0, "alignment");

__device__ __forceinline__ float post_jac(float v, float damping, int clip) {
    v *= damping;
    if (clip) v = fminf(fmaxf(v, -1.0f), 1.0f);
    return v;
}

// write columns 8h..8h+7 of row r of a 128 x 32 K-major swizzled operand as a tf32 pair
__device__ __forceinline__ void put_row_pair(unsigned char *hi, unsigned char *lo, int r, int h,
                                             const float (&v)[kCols]) {
#pragma unroll
    for (int c = 0; c < kCols / 4; c++) {
        float h4[4], l4[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            h4[e] = to_tf32(v[4 * c + e]);
            l4[e] = to_tf32(v[4 * c + e] - h4[e]);
        }
        const uint32_t off = swz128((uint32_t)r, (uint32_t)(kCols * h + 4 * c));
        *reinterpret_cast<float4 *>(hi + off) = make_float4(h4[0], h4[1], h4[2], h4[3]);
        *reinterpret_cast<float4 *>(lo + off) = make_float4(l4[0], l4[1], l4[2], l4[3]);
    }
}

// kCols consecutive 32-bit TMEM columns of the calling thread's lane
static_assert(kCols == 8 || kCols == 16, "column split");
__device__ __forceinline__ void tmem_ldc(uint32_t taddr, float (&v)[kCols]) {
    if constexpr (kCols == 8)
        tmem_ld8(taddr, v);
    else
        tmem_ld16(taddr, v);
}

// Warp-uniform bounded wait (every lane polls; every lane takes the same branch afterwards).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          unsigned int limit) {
    const bool ok = mbar_wait(bar, parity, abort, limit);
    return __all_sync(0xffffffffu, ok);
}

// Arrive once per warp after every lane's shared-memory writes (made visible to the tensor
// core) and TMEM reads are ordered before the warp barrier.
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
    fence_async_smem();
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

template <int P>
using PassC = std::integral_constant<int, P>;

// hi + lo += v without rounding loss (Knuth's two-sum; the error term is carried in lo)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
}

// The hardware approximations of 2^x, 1/x and log2 x (PTX ex2/rcp/lg2 .approx.ftz: one
// special-function instruction each; relative error about 2^-22, subnormals flushed to zero,
// which the callers tolerate: e^-|z| below 2^-126 only rounds 1 + e^-|z| to 1).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ln(p) for p >= 1: the binary exponent is taken exactly and only the mantissa in [1, 2) goes
// through the hardware log2 (absolute error about 2^-22 there)
__device__ __forceinline__ float log_of_product(float p) {
    const int b = __float_as_int(p);
    const float e = (float)((b >> 23) - 127);
    const float mant = __int_as_float((b & 0x007fffff) | 0x3f800000);
    return (e + lg2_approx(mant)) * 0.69314718055994531f;
}

template <typename S_>
__global__ void __launch_bounds__(kThreads, 1) eval_logreg_tc_kernel(EvalArgs A) {
    if (A.skip && *(volatile const int *)A.skip) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const uint32_t sb = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = A.T, D = A.D, N = A.N;
    const bool fused = A.fs_flags != nullptr;
    const int nch = (N + kNB - 1) / kNB;
    const bool want_dh = A.jac == PMCMC_JAC_DIAG;
    // dense Jacobian (assembled by the tensor-core J kernel): the weights sigmoid'(z) at x go to
    // w_out (T x N, FP32), and no diagonal J is written
    const bool want_w = A.jac == PMCMC_JAC_DENSE && A.w_out != nullptr;
    const unsigned int limit = A.spin_limit ? A.spin_limit : kDefaultSpinLimit;
    volatile int *abort_f = reinterpret_cast<volatile int *>(sm + oMisc + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + oMisc);
    auto bar = [&](int i) -> uint32_t { return sb + oBar + 8u * (uint32_t)i; };

    if (tid == 0) {
        for (int i = 0; i < kNumBars; i++) {
            uint32_t cnt = 1;
            if ((i >= bCfull && i < bCfull + 4) || i == bVready) cnt = kEpiWarps;  // one per warp
            if ((i >= bEmpty && i < bEmpty + kStages) || i == bFin) cnt = 2;      // both issuers
            mbar_init(bar(i), cnt);
        }
        *abort_f = 0;
        // the fused Newton update walks back over earlier tiles: tiles are taken by ticket, in
        // dispatch order, so every tile a CTA waits on belongs to a CTA already running
        unsigned int tile_ = blockIdx.x, ep = 0;
        if (fused) {
            tile_ = atomicAdd(&A.fs_ctl->ticket, 1u);
            ep = *(volatile unsigned int *)&A.fs_ctl->epoch;
        }
        reinterpret_cast<unsigned int *>(sm + oMisc)[2] = tile_;
        reinterpret_cast<unsigned int *>(sm + oMisc)[3] = ep;
        fence_barrier_init();
    }
    if (warp == kMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tmem_slot;
    const int tile = (int)reinterpret_cast<const unsigned int *>(sm + oMisc)[2];
    const unsigned int epoch = reinterpret_cast<const unsigned int *>(sm + oMisc)[3];
    const int t0 = tile * kM;

    if (warp == kCopyWarp && lane == kCopyLane) {
        // ---------------- producer: chunk images, both passes ----------------
        {
            const unsigned char *img = static_cast<const unsigned char *>(A.tc_img);
            int k = 0;
            for (; k < 2 * nch; k++) {
                const int s = k % kStages;
                if (k >= kStages && !mbar_wait(bar(bEmpty + s), (uint32_t)((k / kStages) - 1) & 1u, abort_f, limit))
                    break;
                mbar_arrive_expect_tx(bar(bFull + s), kImg);
                bulk_g2s(sb + oStage + s * kStageStride, img + (size_t)(k % nch) * kImg, kImg, bar(bFull + s));
            }
            for (int q = k > kStages ? k - kStages : 0; q < k; q++)
                mbar_wait_drain(bar(bFull + q % kStages), (uint32_t)(q / kStages) & 1u, kDrainLimit);
        }
    } else if (warp == kIssZ) {
        // ---------------- Z = V X^T issue (one thread per product stream) ----------------
        // Issuing from two threads lets the Z and the G products of different chunks overlap.
        // GEMM1 runs kZbuf chunks ahead: Z(k + 3) reuses the buffer of Z(k), which the epilogue
        // has loaded (prefetch) before it signals C(k) ready.
        if (lane == 0) {
            auto issue_z = [&](int k) -> bool {
                const int s = k % kStages;
                if (!mbar_wait(bar(bFull + s), (uint32_t)(k / kStages) & 1u, abort_f, limit)) return false;
                tc_fence_after();
                const uint32_t st = sb + oStage + s * kStageStride;
                const uint32_t zt = tm + kColZ + (uint32_t)(k % kZbuf) * 64u;
#pragma unroll
                for (int kk = 0; kk < 4; kk++) {
                    const uint64_t ah = sdesc(sb + oVhi + 32 * kk), al = sdesc(sb + oVlo + 32 * kk);
                    const uint64_t b2 = sdesc(st + 32 * kk);  // [X_hi; X_lo], 64 rows
                    mma_tf32(zt, al, b2, kIdesc64, kk > 0);
                    mma_tf32(zt, ah, b2, kIdesc64, 1);
                }
                mma_commit(bar(bZfull + k % kZbuf));
                mma_commit(bar(bEmpty + s));  // this issuer is done with the stage
                return true;
            };
            bool ok = true;
            for (int pass = 0; pass < 2 && ok; pass++) {
                ok = mbar_wait(bar(bVready), (uint32_t)pass, abort_f, limit);
                if (!ok) break;
                tc_fence_after();
                const int kb = pass * nch;
                for (int j = 0; j < kZbuf && j < nch && ok; j++) ok = issue_z(kb + j);
                // Z(k) overwrites the buffer of Z(k - 3), which the epilogue loads while it computes
                // chunk k - 4 (in the pass prologue for k - 3 = kb): C(max(k - 4, kb)) ready
                // implies that buffer is free
                for (int k = kb + kZbuf; k < kb + nch && ok; k++) {
                    const int c = k - 4 > kb ? k - 4 : kb;
                    if (!(ok = mbar_wait(bar(bCfull + (c & 3)), (uint32_t)(c >> 2) & 1u, abort_f, limit))) break;
                    tc_fence_after();
                    ok = issue_z(k);
                }
            }
            mma_commit(bar(bFin));
            mbar_wait_drain(bar(bFin), 0, kDrainLimit);
        }
    } else if (warp == kIssG) {
        // ---------------- G = C X and H = W (X.X) issue ----------------
        if (lane == 0) {
            bool ok = true;
            for (int pass = 0; pass < 2 && ok; pass++) {
                const int kb = pass * nch;
                for (int j = 0; j < nch && ok; j++) {
                    const int k = kb + j;
                    if (!(ok = mbar_wait(bar(bCfull + (k & 3)), (uint32_t)(k >> 2) & 1u, abort_f, limit))) break;
                    tc_fence_after();
                    const uint32_t st = sb + oStage + (k % kStages) * kStageStride;
                    const uint32_t cw = sb + oCW + (k & 1) * kCWStride;
                    const uint32_t gt = tm + kColG + (uint32_t)(k & 1) * 64u;  // fresh per chunk
#pragma unroll
                    for (int kk = 0; kk < 4; kk++) {
                        const uint64_t ch = sdesc(cw + 32 * kk), cl = sdesc(cw + kRowOp + 32 * kk);
                        const uint64_t b2 = sdesc(st + 2 * kOp + 32 * kk);  // [X^T_hi; X^T_lo]
                        mma_tf32(gt, cl, b2, kIdesc64, kk > 0 ? 1u : 0u);
                        mma_tf32(gt, ch, b2, kIdesc64, 1);
                    }
                    if (pass == 0 && want_dh) {
#pragma unroll
                        for (int kk = 0; kk < 4; kk++)
                            mma_tf32(tm + kColH, sdesc(cw + 2 * kRowOp + 32 * kk), sdesc(st + 4 * kOp + 32 * kk),
                                     kIdesc, (j > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(bar(bCempty + (k & 1)));
                    mma_commit(bar(bEmpty + k % kStages));
                }
                if (ok) mma_commit(bar(bGdone));
            }
            mma_commit(bar(bFin));
            mbar_wait_drain(bar(bFin), 0, kDrainLimit);
        }
    } else if (warp < kEpiWarps) {
        // ---------------- epilogue warpgroups ----------------
        const int q = warp & 3, h = warp >> 2;
        const int r = q * 32 + lane;
        const int t = t0 + r;
        const bool tv = t < T;
        const int d0 = kCols * h;  // this warpgroup's dimensions d0 .. d0 + 7
        const uint32_t lrow = tm + ((uint32_t)(q * 32) << 16);
        const float eps = (float)A.eps;
        const float inv_sp2 = (float)(1.0 / (A.sigma_p * A.sigma_p));
        // fused mode: the iterate ping-pongs between A.s and A.s_alt with the iteration parity
        const int par = (fused && A.iter) ? (*A.iter & 1) : 0;
        const float *s = static_cast<const float *>(par ? A.s_alt : A.s);
        float *s_next = static_cast<float *>(par ? const_cast<void *>(A.s) : A.s_alt);
        const float *s0 = static_cast<const float *>(A.s0);
        const float *xin = static_cast<const float *>(A.xi);
        // own dimensions of x = s_{t-1} and of the noise, re-read where needed (L2)
        auto load_x = [&](float (&v)[kCols]) {
#pragma unroll
            for (int i = 0; i < kCols; i++) {
                const int d = d0 + i;
                v[i] = (tv && d < D) ? (t == 0 ? s0[d] : s[(size_t)(t - 1) * D + d]) : 0.0f;
            }
        };
        auto load_xi = [&](float (&v)[kCols]) {
#pragma unroll
            for (int i = 0; i < kCols; i++) {
                const int d = d0 + i;
                v[i] = (tv && d < D) ? xin[(size_t)t * D + d] : 0.0f;
            }
        };
        float xt[kCols];              // the proposal (own dimensions)
        float gs[kCols];              // running G sum (own dimensions)
        // own dimensions of x = s_{t-1}, the noise, s_t and X^T y (loaded at each pass end)
        float x[kCols], xv[kCols], sv[kCols], ty[kCols];
        const float *xty = reinterpret_cast<const float *>(static_cast<const unsigned char *>(A.tc_img) +
                                                           (size_t)nch * kImg);
        // -sum softplus partials (own columns) of the two passes, compensated (hi + lo)
        float ll0h = 0.0f, ll0l = 0.0f, ll1h = 0.0f, ll1l = 0.0f;
        bool ok = true;
#pragma unroll
        for (int i = 0; i < kCols; i++) xt[i] = gs[i] = 0.0f;
        load_x(x);
        put_row_pair(sm + oVhi, sm + oVlo, r, h, x);
        warp_arrive(bar(bVready));
        // log u (FP64) while the first products run; read back by the same thread at the end
        if (h == 0) reinterpret_cast<double *>(sm + oLogu)[r] = tv ? log(A.u[t]) : 0.0;
        auto add_partial = [&](int kc) {  // G of chunk kc, own dimensions
            float gp[kCols], gpl[kCols];
            tmem_ldc(lrow + kColG + 64u * (uint32_t)(kc & 1) + (uint32_t)d0, gp);
            tmem_ldc(lrow + kColG + 64u * (uint32_t)(kc & 1) + 32u + (uint32_t)d0, gpl);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < kCols; i++) gs[i] += gp[i] + gpl[i];
        };
        // one pass over the design: chunk loop, then the pass end
        auto run_pass = [&](auto pc) {
            constexpr int pass = decltype(pc)::value;
            constexpr bool kW = pass == 0;  // Hessian weights are needed in pass 1 only
            // software pipeline: Z(k + 1) and the G partial of chunk k - 2 are loaded from TMEM
            // while chunk k is computed from registers
            float zcur[kCols];
            {
                const int k = pass * nch;
                if (ok && (ok = warp_wait(bar(bZfull + k % kZbuf), (uint32_t)(k / kZbuf) & 1u, abort_f, limit))) {
                    tc_fence_after();
                    float zl[kCols];
                    tmem_ldc(lrow + kColZ + (uint32_t)(k % kZbuf) * 64u + (uint32_t)d0, zcur);
                    tmem_ldc(lrow + kColZ + (uint32_t)(k % kZbuf) * 64u + 32u + (uint32_t)d0, zl);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < kCols; i++) zcur[i] += zl[i];
                }
            }
            for (int j = 0; j < nch && ok; j++) {
                const int k = pass * nch + j, b = k & 1, si = k % kStages;
                float znext[kCols], znl[kCols], gp[kCols], gpl[kCols];
                const bool more = j + 1 < nch;
                if (more) {
                    if (!(ok = warp_wait(bar(bZfull + (k + 1) % kZbuf), (uint32_t)((k + 1) / kZbuf) & 1u, abort_f, limit)))
                        break;
                }
                // G of chunk k - 2 is complete: its C buffer is free and its partial readable
                if (k >= 2 && !(ok = warp_wait(bar(bCempty + b), (uint32_t)((k - 2) >> 1) & 1u, abort_f, limit)))
                    break;
                if (!(ok = warp_wait(bar(bFull + si), (uint32_t)(k / kStages) & 1u, abort_f, limit))) break;
                tc_fence_after();
                if (more) {
                    tmem_ldc(lrow + kColZ + (uint32_t)((k + 1) % kZbuf) * 64u + (uint32_t)d0, znext);
                    tmem_ldc(lrow + kColZ + (uint32_t)((k + 1) % kZbuf) * 64u + 32u + (uint32_t)d0, znl);
                }
                const bool part2 = j >= 2;
                if (part2) {
                    tmem_ldc(lrow + kColG + 64u * (uint32_t)(k & 1) + (uint32_t)d0, gp);
                    tmem_ldc(lrow + kColG + 64u * (uint32_t)(k & 1) + 32u + (uint32_t)d0, gpl);
                }
                const float4 *ys4 =
                    reinterpret_cast<const float4 *>(sm + oStage + si * kStageStride + 5 * kOp) + (kCols / 4) * h;
                float yv8[kCols];  // the labels of this warpgroup's columns
#pragma unroll
                for (int c4 = 0; c4 < kCols / 4; c4++) {
                    const float4 yq = ys4[c4];
                    yv8[4 * c4] = yq.x;
                    yv8[4 * c4 + 1] = yq.y;
                    yv8[4 * c4 + 2] = yq.z;
                    yv8[4 * c4 + 3] = yq.w;
                }
                float chi[kCols], clo[kCols], whi[kCols];
                // The log-likelihood enters the MH ratio only as ll(x~) - ll(x), so its part
                // sum_n y_n z_n is taken in the tail as (x~ - x) . X^T y, and here only
                // -sum_n softplus(z_n) = -sum_n max(z_n, 0) - log prod_n (1 + e^-|z_n|).  Padded
                // rows (n >= N) have X_n = 0, hence z = 0, c X_n = 0 and w X_n.X_n = 0, and a
                // log 2 that is the same in both passes: no masking is needed.
                float negrelu = 0.0f, prod = 1.0f;
#pragma unroll
                for (int i = 0; i < kCols; i++) {
                    const float zz = zcur[i];
                    const float m = ex2_approx(fabsf(zz) * -1.4426950408889634f);  // e^-|z|
                    const float onep = 1.0f + m;
                    const float qv = rcp_approx(onep);
                    const float mq = m * qv;
                    const bool pos = zz >= 0.0f;
                    const float p = pos ? qv : mq;   // sigmoid(z)
                    const float c = yv8[i] - p;
                    negrelu -= fmaxf(zz, 0.0f);
                    prod *= onep;
                    // c = c_hi + c_lo exactly; the tensor core drops the low 13 bits of c_lo
                    // (below 2^-20 |c|) and of w
                    chi[i] = tf32_trunc(c);
                    clo[i] = c - chi[i];
                    if (kW) whi[i] = p * (pos ? mq : qv);  // sigmoid'(z)
                }
                const float llc = negrelu - log_of_product(prod);
                if (pass) two_sum_acc(ll1h, ll1l, llc);
                else two_sum_acc(ll0h, ll0l, llc);
                unsigned char *cw = sm + oCW + b * kCWStride;
#pragma unroll
                for (int c4 = 0; c4 < kCols / 4; c4++) {
                    const uint32_t off = swz128((uint32_t)r, (uint32_t)(d0 + 4 * c4));
                    *reinterpret_cast<float4 *>(cw + off) =
                        make_float4(chi[4 * c4], chi[4 * c4 + 1], chi[4 * c4 + 2], chi[4 * c4 + 3]);
                    *reinterpret_cast<float4 *>(cw + kRowOp + off) =
                        make_float4(clo[4 * c4], clo[4 * c4 + 1], clo[4 * c4 + 2], clo[4 * c4 + 3]);
                    if (kW && want_dh)
                        *reinterpret_cast<float4 *>(cw + 2 * kRowOp + off) =
                            make_float4(whi[4 * c4], whi[4 * c4 + 1], whi[4 * c4 + 2], whi[4 * c4 + 3]);
                }
                if (kW && want_w && tv) {
                    float *wr = static_cast<float *>(A.w_out) + (size_t)t * N + (size_t)j * kNB + d0;
#pragma unroll
                    for (int i = 0; i < kCols; i++)
                        if (j * kNB + d0 + i < N) wr[i] = whi[i];
                }
                tmem_wait_ld();
                if (part2) {
#pragma unroll
                    for (int i = 0; i < kCols; i++) gs[i] += gp[i] + gpl[i];
                }
                if (more) {
#pragma unroll
                    for (int i = 0; i < kCols; i++) zcur[i] = znext[i] + znl[i];
                }
                warp_arrive(bar(bCfull + (k & 3)));
            }
            // pass end: the last one or two partials complete G of this pass.  The global loads
            // the pass end and the tail need (x, the noise; s_t and X^T y after pass 2) are issued
            // before the wait, so their latency overlaps the last products.
            load_x(x);
            load_xi(xv);
            if (pass == 1) {
#pragma unroll
                for (int i = 0; i < kCols; i++) {
                    sv[i] = (tv && d0 + i < D) ? s[(size_t)t * D + d0 + i] : 0.0f;
                    ty[i] = xty[d0 + i];
                }
            }
            if (ok && (ok = warp_wait(bar(bGdone), (uint32_t)pass, abort_f, limit))) {
                tc_fence_after();
                const int kb = pass * nch;
                if (nch >= 2) add_partial(kb + nch - 2);
                add_partial(kb + nch - 1);
                if (pass == 0) {
                    // the proposal x~ = x + eps grad log p(x) + sqrt(2 eps) xi (own dimensions)
                    const float sq = sqrtf(2.0f * eps);
#pragma unroll
                    for (int i = 0; i < kCols; i++)
                        xt[i] = d0 + i < D ? x[i] + eps * (gs[i] - x[i] * inv_sp2) + sq * xv[i] : 0.0f;
                    put_row_pair(sm + oVhi, sm + oVlo, r, h, xt);
                    warp_arrive(bar(bVready));
#pragma unroll
                    for (int i = 0; i < kCols; i++) gs[i] = 0.0f;
                }
            }
        };
        run_pass(PassC<0>{});
        run_pass(PassC<1>{});
        // gs holds the own dimensions of the G row at x~.  The MH log-ratio (FP64):
        //   ell = [ll(x~) - |x~|^2/2sp2] - [ll(x) - |x|^2/2sp2] - |e|^2/(4 eps) + |xi|^2/2,
        //   e = x - x~ - eps grad log p(x~), summed over the four warpgroups.
        // The per-dimension terms of the log-ratio are formed in FP32 from the FP32 state, the
        // proposal and the gradient (their rounding, ~1e-7 each, is far below what the FP32
        // states themselves carry into ell); the log-likelihood difference, which cancels two
        // sums of N terms, and the sum over the warpgroups are FP64.  Every global load of the
        // tail (x = s_{t-1}, the noise, s_t) is issued before any of them is used.
        double *part = reinterpret_cast<double *>(sm + oPart);
        int *accf = reinterpret_cast<int *>(sm + oAcc);
        {
            const float inv2sp2 = 0.5f * inv_sp2, inv4e = 0.25f / eps;
            float qf = 0.0f;
#pragma unroll
            for (int i = 0; i < kCols; i++) {
                if (d0 + i < D) {
                    const float g2 = gs[i] - xt[i] * inv_sp2;
                    const float e = x[i] - xt[i] - eps * g2;
                    qf += (xt[i] - x[i]) * ty[i] - (xt[i] - x[i]) * (xt[i] + x[i]) * inv2sp2 -
                          e * e * inv4e + 0.5f * xv[i] * xv[i];
                }
            }
            part[h * kM + r] = (((double)ll1h - (double)ll0h) + ((double)ll1l - (double)ll0l)) + (double)qf;
        }
        named_bar(1, kEpiThreads);
        const bool valid = tv && ok && !*abort_f;
        double margin = INFINITY;
        int acc_i = 0;
        if (h == 0) {
            int acc = 0;
            if (valid) {
                double ell = part[r];
#pragma unroll
                for (int hg = 1; hg < kGroups; hg++) ell += part[hg * kM + r];
                const double la = (ell < 0.0 || isnan(ell)) ? ell : 0.0;
                const double gtl = la - reinterpret_cast<const double *>(sm + oLogu)[r];
                acc = gtl > 0.0;
                margin = fabs(gtl);
                acc_i = acc;
                if (A.ell_out) A.ell_out[t] = ell;
                if (A.acc_out) A.acc_out[t] = acc ? 1 : 0;
            }
            accf[r] = acc;
        }
        named_bar(1, kEpiThreads);
        float err = -INFINITY, rmax = 0.0f;
        float dh[kCols];
#pragma unroll
        for (int i = 0; i < kCols; i++) dh[i] = 0.0f;
        if (want_dh && ok) {
            // diag(X^T W X) accumulated over the chunks of pass 1 (untouched by pass 2); the
            // condition is warp-uniform, as the collective TMEM load requires
            tmem_ldc(lrow + kColH + (uint32_t)d0, dh);
            tmem_wait_ld();
        }
        const float rtolf = (float)A.rtol;
        float fa[kCols], fb[kCols];  // the scan pair (J_t, r_t) of each own dimension; identity if unused
#pragma unroll
        for (int i = 0; i < kCols; i++) {
            fa[i] = 1.0f;
            fb[i] = 0.0f;
        }
        if (valid) {
            const bool acc = accf[r] != 0;
            S_ *bout = static_cast<S_ *>(A.b_out);
            S_ *aout = static_cast<S_ *>(A.a_out);
            float *fout = static_cast<float *>(A.f_out);
            const float damping = (float)A.damping;
#pragma unroll
            for (int i = 0; i < kCols; i++) {
                const int d = d0 + i;
                if (d < D) {
                    const size_t o = (size_t)t * D + d;
                    const float f = acc ? xt[i] : x[i];
                    const float rr = f - sv[i];
                    const float ar = fabsf(rr);
                    const float ee = ar - rtolf * fabsf(sv[i]);
                    err = isnan(ee) ? INFINITY : fmaxf(err, ee);
                    rmax = isnan(ar) ? INFINITY : fmaxf(rmax, ar);
                    float jv = 0.0f;
                    if (want_dh) jv = post_jac(acc ? 1.0f + eps * (-dh[i] - inv_sp2) : 1.0f, damping, A.clip);
                    if (bout) store_as<S_, float>(bout + o, rr);
                    if (fout) fout[o] = f;
                    if (aout && !want_w) store_as<S_, float>(aout + o, jv);
                    fa[i] = jv;
                    fb[i] = rr;
                }
            }
        }
        float dmx = 0.0f;        // fused update: max |delta| and non-finite resets of own elements
        unsigned int nres = 0;
        if (fused) {
            // Newton update of this tile (Eq. 3 in delta form): delta_t = J_t delta_{t-1} + r_t
            // over the 128 timesteps, carried in from the earlier tiles, and s_t + delta_t
            // written to the other iterate buffer.  Lanes are timesteps, so a warp scans its 32
            // timesteps of 8 channels with shuffles; warp totals compose across the four warps
            // of a warpgroup into the tile aggregate, which is published.  The carry into the tile
            // composes the aggregates of all earlier tiles (published independently of any
            // carry, so no tile waits on another's carry): warp w composes a segment of them,
            // warp 0 folds the 16 segments.
            float *wtot = reinterpret_cast<float *>(sm + oFw);    // [warp][channel][A, B]
            float *pre = reinterpret_cast<float *>(sm + oFpre);   // [q][32] A, then [q][32] B
            float *segm = reinterpret_cast<float *>(sm + oFseg);  // [16 segments][32][A, B]
            float *car = reinterpret_cast<float *>(sm + oFcar);   // [32]
            float IA[kCols], IB[kCols];
#pragma unroll
            for (int i = 0; i < kCols; i++) {
                IA[i] = fa[i];
                IB[i] = fb[i];
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int i = 0; i < kCols; i++) {
                    const float pa = __shfl_up_sync(0xffffffffu, IA[i], off);
                    const float pb = __shfl_up_sync(0xffffffffu, IB[i], off);
                    if (lane >= off) {
                        IB[i] = IA[i] * pb + IB[i];
                        IA[i] = IA[i] * pa;
                    }
                }
            }
            if (lane == 31) {
#pragma unroll
                for (int i = 0; i < kCols; i++) {
                    wtot[(warp * kCols + i) * 2] = IA[i];
                    wtot[(warp * kCols + i) * 2 + 1] = IB[i];
                }
            }
            named_bar(1, kEpiThreads);
            if (tid < kDP) {  // channel tid = 8 h' + i': compose warps 4 h' .. 4 h' + 3
                const int hh = tid / kCols, ii = tid % kCols;
                float PA = 1.0f, PB = 0.0f;
#pragma unroll
                for (int qq = 0; qq < 4; qq++) {
                    pre[qq * 32 + tid] = PA;
                    pre[128 + qq * 32 + tid] = PB;
                    const float WA = wtot[((4 * hh + qq) * kCols + ii) * 2];
                    const float WB = wtot[((4 * hh + qq) * kCols + ii) * 2 + 1];
                    PB = WA * PB + WB;
                    PA = WA * PA;
                }
                A.fs_agg[((size_t)tile * 2) * kDP + tid] = PA;
                A.fs_agg[((size_t)tile * 2 + 1) * kDP + tid] = PB;
                __threadfence();
            }
            __syncwarp();
            if (tid == 0) st_release(A.fs_flags + tile, make_flag(epoch, kFlagAgg));
            // segment of warp w: tiles [w per, (w + 1) per) below this tile; lane = channel
            {
                const int per = (tile + kEpiWarps - 1) / kEpiWarps;
                const int j0 = warp * per, j1 = min(tile, j0 + per);
                float SA = 1.0f, SB = 0.0f;
                for (int jb = j0; jb < j1; jb += 32) {
                    const int nj = min(32, j1 - jb);
                    if (lane < nj) wait_flag(A.fs_flags, jb + lane, epoch, limit, A.fs_ctl);
                    __syncwarp();
                    for (int jc = 0; jc < nj; jc += 8) {
                        float ga[8], gb[8];
#pragma unroll
                        for (int u = 0; u < 8; u++) {
                            const int j = jb + jc + u;
                            const bool on = jc + u < nj;
                            ga[u] = on ? __ldcg(A.fs_agg + ((size_t)j * 2) * kDP + lane) : 1.0f;
                            gb[u] = on ? __ldcg(A.fs_agg + ((size_t)j * 2 + 1) * kDP + lane) : 0.0f;
                        }
#pragma unroll
                        for (int u = 0; u < 8; u++) {  // later tiles on the left
                            SB = ga[u] * SB + gb[u];
                            SA = ga[u] * SA;
                        }
                    }
                }
                segm[(warp * 32 + lane) * 2] = SA;
                segm[(warp * 32 + lane) * 2 + 1] = SB;
            }
            named_bar(1, kEpiThreads);
            if (warp == 0) {
                float c = 0.0f;  // the carry into tile 0 is zero
#pragma unroll
                for (int w = 0; w < kEpiWarps; w++)
                    c = segm[(w * 32 + lane) * 2] * c + segm[(w * 32 + lane) * 2 + 1];
                car[lane] = c;
            }
            named_bar(1, kEpiThreads);
#pragma unroll
            for (int i = 0; i < kCols; i++) {
                const int d = d0 + i;
                const float cq = pre[q * 32 + d] * car[d] + pre[128 + q * 32 + d];  // delta before warp q
                const float dl = IA[i] * cq + IB[i];
                if (valid && d < D) {
                    float sn = sv[i] + dl;
                    if (!isfinite(sn)) {
                        sn = s0[d];
                        nres++;
                    } else {
                        dmx = fmaxf(dmx, fabsf(dl));
                    }
                    s_next[(size_t)t * D + d] = sn;
                }
            }
        }
        if (A.stats) {
            // residuals, margins and update sizes are reduced as FP32 (the residual is an FP32
            // quantity; the margin is a diagnostic), decisions and resets as integers
            float *red = reinterpret_cast<float *>(sm + oRed);
            const float e1 = warp_max(err), e2 = warp_max(rmax), e3 = warp_min((float)margin);
            const int e4 = __reduce_add_sync(0xffffffffu, acc_i);
            const float e5 = warp_max(dmx);
            const unsigned int e6 = __reduce_add_sync(0xffffffffu, nres);
            if (lane == 0) {
                red[8 * warp + 0] = e1;
                red[8 * warp + 1] = e2;
                red[8 * warp + 2] = e3;
                reinterpret_cast<int *>(red)[8 * warp + 3] = e4;
                red[8 * warp + 4] = e5;
                reinterpret_cast<unsigned int *>(red)[8 * warp + 5] = e6;
            }
            named_bar(1, kEpiThreads);
            if (tid == 0) {
                float m1 = red[0], m2 = red[1], m3 = red[2], m5 = red[4];
                int m4 = reinterpret_cast<int *>(red)[3];
                unsigned int m6 = reinterpret_cast<unsigned int *>(red)[5];
                for (int w = 1; w < kEpiWarps; w++) {
                    m1 = fmaxf(m1, red[8 * w]);
                    m2 = fmaxf(m2, red[8 * w + 1]);
                    m3 = fminf(m3, red[8 * w + 2]);
                    m4 += reinterpret_cast<int *>(red)[8 * w + 3];
                    m5 = fmaxf(m5, red[8 * w + 4]);
                    m6 += reinterpret_cast<unsigned int *>(red)[8 * w + 5];
                }
                atomic_max_d(&A.stats->err, (double)m1);
                atomic_max_d(&A.stats->rmax, (double)m2);
                atomic_min_d(&A.stats->min_margin, (double)m3);
                if (m4 > 0) atomicAdd(&A.stats->accepts, (unsigned long long)m4);
                if (m5 > 0.0f) atomic_max_d(&A.stats->dmax, (double)m5);
                if (m6) atomicAdd(&A.stats->resets, (unsigned long long)m6);
            }
        }
        if (fused) {
            // the last tile to finish resets the ticket and advances the epoch for the next launch
            named_bar(1, kEpiThreads);
            if (tid == 0) {
                if (*abort_f && A.timeout) atomicExch(A.timeout, 1u);  // before counting out
                __threadfence();
                const unsigned int dn = atomicAdd(&A.fs_ctl->done, 1u);
                if (dn == gridDim.x - 1) {
                    A.fs_ctl->ticket = 0;
                    A.fs_ctl->done = 0;
                    A.fs_ctl->epoch = A.fs_ctl->epoch + 1u;
                    __threadfence();
                    // every tile's statistics (and timeout) were published before it counted
                    // out: the loop's decision for this iteration can be taken here
                    if (A.loop)
                        loop_control_step(A.loop, (cudaGraphConditionalHandle)A.loop_handle, A.loop_atol,
                                          A.loop_max_iters);
                }
            }
        }
    }
    __syncwarp();  // the issuer and producer lanes of a warp re-converge here
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tm, kTmemCols);
    }
    if (tid == 0 && *abort_f && A.timeout) atomicExch(A.timeout, 1u);
}

// Chunk images of the design: per chunk of 32 rows, the tf32 pair of X (rows n, columns d),
// the tf32 pair of X^T (rows d, columns n), tf32 of (X.X)^T, and the 32 labels; each operand
// block already in the swizzled shared-memory layout, so one bulk copy stages a chunk.
__global__ void logreg_tc_pack_kernel(const float *__restrict__ X, const float *__restrict__ y, int N, int D,
                                      unsigned char *__restrict__ img) {
    unsigned char *base = img + (size_t)blockIdx.x * kImg;
    for (int e = threadIdx.x; e < kNB * kDP; e += blockDim.x) {
        const int nl = e / kDP, d = e % kDP;
        const int n = blockIdx.x * kNB + nl;
        const float v = (n < N && d < D) ? X[(size_t)n * D + d] : 0.0f;
        const float hi = to_tf32(v), lo = to_tf32(v - hi);
        *reinterpret_cast<float *>(base + 0 * kOp + swz128(nl, d)) = hi;
        *reinterpret_cast<float *>(base + 1 * kOp + swz128(nl, d)) = lo;
        *reinterpret_cast<float *>(base + 2 * kOp + swz128(d, nl)) = hi;
        *reinterpret_cast<float *>(base + 3 * kOp + swz128(d, nl)) = lo;
        *reinterpret_cast<float *>(base + 4 * kOp + swz128(d, nl)) = to_tf32(v * v);
    }
    if (threadIdx.x < kNB) {
        const int n = blockIdx.x * kNB + threadIdx.x;
        reinterpret_cast<float *>(base + 5 * kOp)[threadIdx.x] = n < N ? y[n] : 0.0f;
    }
}

}  // namespace

bool logreg_tc_supported(const EvalArgs &A) {
    return !A.f64 && A.engine == 0 && A.target == PMCMC_LOGREG && A.sampler == PMCMC_MALA && A.D >= 1 &&
           A.D <= kDP && A.N >= 1 &&
           (A.jac == PMCMC_JAC_ZERO ||
            ((A.jac == PMCMC_JAC_DIAG || A.jac == PMCMC_JAC_DENSE) && A.gate_grad == 0));
}

// the chunk images, then X^T y (kDP floats)
size_t logreg_tc_image_bytes(int N) { return (size_t)ceil_div(N, kNB) * kImg + kDP * sizeof(float); }

// X^T y (FP64 sums, rounded once), after the chunk images; padded dimensions are zero.  One
// CTA per dimension.
__global__ void logreg_tc_xty_kernel(const float *__restrict__ X, const float *__restrict__ y, int N, int D,
                                     float *__restrict__ xty) {
    __shared__ double part[8];
    const int d = blockIdx.x;
    double acc = 0.0;
    if (d < D)
        for (int n = threadIdx.x; n < N; n += blockDim.x) acc += (double)y[n] * (double)X[(size_t)n * D + d];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        xty[d] = (float)t;
    }
}

cudaError_t launch_logreg_tc_pack(const void *X, const void *y, int N, int D, void *img, cudaStream_t st) {
    if (N <= 0 || D > kDP) return cudaErrorInvalidValue;
    logreg_tc_pack_kernel<<<ceil_div(N, kNB), 256, 0, st>>>(static_cast<const float *>(X),
                                                           static_cast<const float *>(y), N, D,
                                                           static_cast<unsigned char *>(img));
    logreg_tc_xty_kernel<<<kDP, 256, 0, st>>>(static_cast<const float *>(X), static_cast<const float *>(y), N, D,
                                            reinterpret_cast<float *>(static_cast<unsigned char *>(img) +
                                                                      (size_t)ceil_div(N, kNB) * kImg));
    return cudaGetLastError();
}

cudaError_t launch_eval_logreg_tc(const EvalArgs &A, cudaStream_t st) {
    if (!A.tc_img || reinterpret_cast<uintptr_t>(A.tc_img) % 16 != 0) return cudaErrorInvalidValue;
    if (A.T <= 0) return cudaSuccess;
    static bool attr_set[2] = {false, false};
    const int which = A.bf16 ? 1 : 0;
    auto k = A.bf16 ? eval_logreg_tc_kernel<__nv_bfloat16> : eval_logreg_tc_kernel<float>;
    if (!attr_set[which]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set[which] = true;
    }
    k<<<ceil_div(A.T, kM), kThreads, kSmemBytes, st>>>(A);
    return cudaGetLastError();
}

}  // namespace pm
