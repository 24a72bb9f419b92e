// Dense Jacobians of held-decision MALA steps on the logistic target, on the tensor cores.
//
// For the adjoint (the reverse recursion of the fixed point with the decisions held), every
// accepted step t needs J_t = I + eps H(x_t) with x_t = s_{t-1} and
//   H(x) = -X^T diag(w) X - I / sigma_p^2,   w_n = sigmoid(z_n) (1 - sigmoid(z_n)),   z = X x,
// an N x D x D contraction per step: the dominant work of the adjoint (Section 3.4's MALA
// Jacobian with the gate held; the reverse recursion itself is D^3 per step).  This file forms
// it for 64 < D <= 128 as a tcgen05 product with FP32 accuracy:
//
//   Acc[i][(u, j)] = sum_n A[i][n] B[(u, j)][n],   A[i][n] = X[n][i],   B[(u, j)][n] = w_u[n] X[n][j]
//
// M = 128 rows i (D zero-padded), N = 256 = two steps u x 128 columns j, K = the N data rows in
// chunks of 32.  Both operands are split into a tf32 head (x truncated to tf32) and a
// remainder, and the product is hi.hi + hi.lo + lo.hi (three kind::tf32 MMAs per K-step).  A
// comes from a pre-swizzled image of X^T streamed by bulk copies, its remainder stored exactly
// (hi + lo = x); B is formed per chunk by CUDA-core warps from the same image scaled by w,
// which they compute for the chunk's 32 rows from the image and the two states, its remainder
// rounded to the nearest tf32.  The tensor core's FP32 accumulation truncates, so
// it is kept short: two TMEM accumulators alternate every kPeriod chunks and the worker warps
// drain each finished one into registers (round-to-nearest sums), so no accumulator sees more
// than 12 kPeriod additions.
//
// Roles (one CTA per SM, persistent over pairs of listed steps): 16 worker warps (w, B
// formation, accumulator drains, the J write), one MMA-issuing thread, one bulk-copy thread.
// Every wait is bounded: on timeout the CTA raises its abort flag, the roles stop, in-flight
// copies and MMAs are drained, TMEM is freed and the timeout word is set.
#include <cuda_runtime.h>

#include "common.cuh"
#include "hess_tc.h"
#include "internal.h"
#include "tc.cuh"

namespace pm {
namespace {

using namespace tc;

constexpr int kM = 128;                  // rows i (and j) of one step's H, D padded
constexpr int kNB = 32;                  // data rows per K-chunk
constexpr int kTile = kM * kNB * 4;      // one 128 x 32 tf32 operand: 16384 bytes
constexpr int kChunk = 2 * kTile;        // image chunk: X^T hi, X^T lo
constexpr int kStages = 4;
constexpr int kPeriod = 1;               // chunks per TMEM accumulator before it is drained
constexpr int kWorkWarps = 16, kWorkThreads = 32 * kWorkWarps;
constexpr int kIssWarp = kWorkWarps, kCopyWarp = kWorkWarps + 1;
constexpr int kThreads = 32 * (kWorkWarps + 2);
constexpr uint32_t kIdesc = idesc_tf32(kM, 2 * kM);
constexpr uint32_t kTmemCols = 512;      // two accumulators of 256 columns
constexpr unsigned int kDrainLimit = 1u << 20;

// shared-memory map (offsets from a 1024-aligned base)
constexpr int oStage = 0;
constexpr int oB = oStage + kStages * kChunk;     // B hi (256 rows), then B lo
constexpr int oXs = oB + 4 * kTile;               // float [2][128]: the two states
constexpr int oZp = oXs + 2 * kM * 4;             // float [2][8][32]: partial z
constexpr int oW = oZp + 2 * 8 * kNB * 4;         // float [2][32]: w of the chunk
constexpr int bFull = 0, bEmpty = kStages, bBready = 2 * kStages, bBfree = bBready + 2,
              bAccFull = bBfree + 2, bAccEmpty = bAccFull + 2, bFin = bAccEmpty + 2,
              kNumBars = bFin + 1;
constexpr int oBar = oW + 2 * kNB * 4;
constexpr int oMisc = oBar + 8 * kNumBars;        // tmem address, abort flag
constexpr int kSmemUsed = oMisc + 16;
constexpr int kSmemBytes = kSmemUsed + 1024;      // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(oB % 1024 == 0 && kChunk % 1024 == 0 && oBar % 8 == 0, "alignment");

__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          unsigned int limit) {
    const bool ok = mbar_wait(bar, parity, abort, limit);
    return __all_sync(0xffffffffu, ok);
}

// one arrival per warp, after the warp's shared-memory writes are visible to the tensor core
// and its TMEM reads are ordered before the barrier
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
    fence_async_smem();
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// Image of X^T for the MMA's A operand: chunk c holds rows n = 32c .. 32c + 31 as a 128 x 32
// K-major 128-byte-swizzled operand (row i = feature, zero beyond D and N), head then remainder.
__global__ void hess_tc_pack_kernel(const float *__restrict__ X, int N, int D, int nch,
                                    unsigned char *__restrict__ img) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (chunk, i, n')
    if (e >= nch * kM * kNB) return;
    const int c = e / (kM * kNB), r = e % (kM * kNB), i = r / kNB, nn = r % kNB;
    const int n = c * kNB + nn;
    const float x = (n < N && i < D) ? X[(size_t)n * D + i] : 0.0f;
    const float hi = tf32_trunc(x);
    unsigned char *base = img + (size_t)c * kChunk;
    const uint32_t off = swz128((uint32_t)i, (uint32_t)nn);
    *reinterpret_cast<float *>(base + off) = hi;
    *reinterpret_cast<float *>(base + kTile + off) = x - hi;  // exact: hi + lo = x
}

__global__ void __launch_bounds__(kThreads, 1)
hess_logreg_tc_kernel(int nlist, const int *__restrict__ list, int D, int N,
                      const unsigned char *__restrict__ img, const float *__restrict__ s0,
                      const float *__restrict__ s, float eps, float inv_sp2, float *__restrict__ Jbuf,
                      unsigned int *timeout, unsigned int limit) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const uint32_t sb = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (N + kNB - 1) / kNB;
    const int nper = (nch + kPeriod - 1) / kPeriod;       // accumulator periods per pair
    const int npairs = (nlist + 1) / 2;
    volatile int *abort_f = reinterpret_cast<volatile int *>(sm + oMisc + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + oMisc);
    auto bar = [&](int i) -> uint32_t { return sb + oBar + 8u * (uint32_t)i; };

    if (tid == 0) {
        for (int i = 0; i < kNumBars; i++) {
            uint32_t cnt = 1;
            if (i == bBready || i == bBready + 1 || i == bAccEmpty || i == bAccEmpty + 1) cnt = kWorkWarps;
            mbar_init(bar(i), cnt);
        }
        *abort_f = 0;
        fence_barrier_init();
    }
    if (warp == kIssWarp) {
        tmem_alloc(smem_u32(tmem_slot), kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tmem_slot;

    if (warp == kCopyWarp) {
        // ---------------- bulk copies of the image chunks, pair after pair ----------------
        if (lane == 0) {
            int k = 0;
            bool ok = true;
            for (int pr = blockIdx.x; pr < npairs && ok; pr += gridDim.x) {
                for (int c = 0; c < nch; c++, k++) {
                    const int st = k % kStages;
                    if (k >= kStages &&
                        !(ok = mbar_wait(bar(bEmpty + st), (uint32_t)((k / kStages) - 1) & 1u, abort_f, limit)))
                        break;
                    mbar_arrive_expect_tx(bar(bFull + st), kChunk);
                    bulk_g2s(sb + oStage + st * kChunk, img + (size_t)c * kChunk, kChunk, bar(bFull + st));
                }
            }
            // copies still in flight complete on their own: wait for them before the CTA exits
            for (int q = k > kStages ? k - kStages : 0; q < k; q++)
                mbar_wait_drain(bar(bFull + q % kStages), (uint32_t)(q / kStages) & 1u, kDrainLimit);
        }
    } else if (warp == kIssWarp) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            int k = 0, gp = 0;  // chunks and accumulator periods issued so far (all pairs)
            bool ok = true;
            for (int pr = blockIdx.x; pr < npairs && ok; pr += gridDim.x) {
                for (int c = 0; c < nch && ok; c++, k++) {
                    const int p = gp + c / kPeriod;
                    const bool first_in_period = (c % kPeriod) == 0;
                    if (first_in_period && p >= 2 &&
                        !(ok = mbar_wait(bar(bAccEmpty + (p & 1)), (uint32_t)((p - 2) >> 1) & 1u, abort_f, limit)))
                        break;
                    const int st = k % kStages;
                    if (!(ok = mbar_wait(bar(bFull + st), (uint32_t)(k / kStages) & 1u, abort_f, limit))) break;
                    const uint32_t acc = tm + (uint32_t)(p & 1) * 256u;
                    const uint32_t a0 = sb + oStage + st * kChunk;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        if (!(ok = mbar_wait(bar(bBready + h), (uint32_t)k & 1u, abort_f, limit))) break;
                        tc_fence_after();
#pragma unroll
                        for (int kk = 2 * h; kk < 2 * h + 2; kk++) {
                            const uint64_t ah = sdesc(a0 + 32 * kk), al = sdesc(a0 + kTile + 32 * kk);
                            const uint64_t bh = sdesc(sb + oB + 32 * kk), bl = sdesc(sb + oB + 2 * kTile + 32 * kk);
                            mma_tf32(acc, ah, bh, kIdesc, (first_in_period && kk == 0) ? 0u : 1u);
                            mma_tf32(acc, ah, bl, kIdesc, 1u);
                            mma_tf32(acc, al, bh, kIdesc, 1u);
                        }
                        mma_commit(bar(bBfree + h));
                    }
                    if (!ok) break;
                    mma_commit(bar(bEmpty + st));
                    if ((c % kPeriod) == kPeriod - 1 || c == nch - 1) mma_commit(bar(bAccFull + (p & 1)));
                }
                gp += nper;
            }
            mma_commit(bar(bFin));
            mbar_wait_drain(bar(bFin), 0, kDrainLimit);
        }
    } else {
        // ---------------- workers ----------------
        const int q = warp & 3, cg = warp >> 2;       // TMEM lane quarter, 64-column group
        const int i_row = 32 * q + lane;               // row i of H held by this thread
        const int u_out = cg >> 1, j0 = (cg & 1) * 64; // its step and first column j
        const uint32_t lrow = tm + ((uint32_t)(32 * q) << 16) + (uint32_t)(cg * 64);
        float *xs = reinterpret_cast<float *>(sm + oXs);
        float *zp = reinterpret_cast<float *>(sm + oZp);
        float *wv = reinterpret_cast<float *>(sm + oW);
        // Named barriers among the worker warps are never skipped by a subset of them: a failed
        // wait marks the warp's status, the next and-barrier makes the status common to all
        // workers, and only then do they leave together.
        int k = 0, gp = 0;
        for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
            // the previous pair's readers of xs passed the and-barrier that ended that pair
            if (tid < 2 * kM) {
                const int u = tid / kM, i = tid % kM, g = 2 * pr + u;
                float v = 0.0f;
                if (g < nlist && i < D) {
                    const int t = list[g];
                    v = t == 0 ? s0[i] : s[(size_t)(t - 1) * D + i];
                }
                xs[tid] = v;
            }
            named_bar(1, kWorkThreads);
            float acc[64];
#pragma unroll
            for (int e = 0; e < 64; e++) acc[e] = 0.0f;
            bool good = true;  // this warp's status (warp-uniform)
            // add accumulator period p into acc (this warp's 64 columns), then release it
            auto drain = [&](int p) -> bool {
                if (!warp_wait(bar(bAccFull + (p & 1)), (uint32_t)(p >> 1) & 1u, abort_f, limit)) return false;
                tc_fence_after();
                const uint32_t a = lrow + (uint32_t)(p & 1) * 256u;
#pragma unroll
                for (int b4 = 0; b4 < 4; b4++) {
                    float v[16];
                    tmem_ld16(a + 16u * b4, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 16; e++) acc[16 * b4 + e] += v[e];
                }
                warp_arrive(bar(bAccEmpty + (p & 1)));
                return true;
            };
            bool all_ok = true;
            for (int c = 0; c < nch; c++, k++) {
                const int st = k % kStages;
                const unsigned char *stg = sm + oStage + st * kChunk;
                good = good && warp_wait(bar(bFull + st), (uint32_t)(k / kStages) & 1u, abort_f, limit);
                // partial z of (step u, row n) over 16 features: warp -> (u, slice), lane -> n
                if (good) {
                    const int u = warp >> 3, sl = warp & 7;
                    float part = 0.0f;
#pragma unroll
                    for (int r = 0; r < 16; r++) {
                        const int i = 16 * sl + r;
                        const uint32_t off = swz128((uint32_t)i, (uint32_t)lane);
                        const float x = *reinterpret_cast<const float *>(stg + off) +
                                        *reinterpret_cast<const float *>(stg + kTile + off);
                        part = fmaf(x, xs[u * kM + i], part);
                    }
                    zp[(u * 8 + sl) * kNB + lane] = part;
                }
                if (!(all_ok = named_bar_and(1, kWorkThreads, good))) break;
                if (tid < 2 * kNB) {
                    const int u = tid / kNB, n = tid % kNB;
                    float z = 0.0f;
#pragma unroll
                    for (int sl = 0; sl < 8; sl++) z += zp[(u * 8 + sl) * kNB + n];
                    const float sg = 1.0f / (1.0f + expf(-z));
                    wv[tid] = (c * kNB + n < N) ? sg * (1.0f - sg) : 0.0f;
                }
                named_bar(1, kWorkThreads);
                // B = w (.) X^T for both steps; half h = K-steps 2h, 2h + 1 (16-byte chunks 4h..4h+3)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    if (good && k >= 1) good = warp_wait(bar(bBfree + h), (uint32_t)(k - 1) & 1u, abort_f, limit);
                    if (!good) continue;
#pragma unroll
                    for (int rep = 0; rep < 2; rep++) {
                        const int pos = tid + rep * kWorkThreads;  // 0 .. 1023
                        const int row = pos >> 2, c4 = 4 * h + (pos & 3);
                        const int u = row >> 7, j = row & (kM - 1);
                        const uint32_t off = swz128((uint32_t)j, (uint32_t)(4 * c4));
                        const float4 xh = *reinterpret_cast<const float4 *>(stg + off);
                        const float4 xl = *reinterpret_cast<const float4 *>(stg + kTile + off);
                        const float4 w4 = *reinterpret_cast<const float4 *>(wv + u * kNB + 4 * c4);
                        float v[4] = {w4.x * (xh.x + xl.x), w4.y * (xh.y + xl.y), w4.z * (xh.z + xl.z),
                                      w4.w * (xh.w + xl.w)};
                        float hv[4], lv[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            hv[e] = tf32_trunc(v[e]);
                            lv[e] = to_tf32(v[e] - hv[e]);
                        }
                        const uint32_t bo = (uint32_t)(u * kTile) + off;
                        *reinterpret_cast<float4 *>(sm + oB + bo) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<float4 *>(sm + oB + 2 * kTile + bo) = make_float4(lv[0], lv[1], lv[2], lv[3]);
                    }
                    warp_arrive(bar(bBready + h));
                }
                // the previous period's accumulator completes behind this chunk's queued MMAs
                if (good && c > 0 && (c % kPeriod) == 0) good = drain(gp + c / kPeriod - 1);
            }
            if (all_ok && good) good = drain(gp + nper - 1);
            gp += nper;
            if (!named_bar_and(1, kWorkThreads, all_ok && good)) break;
            // J_u = I + eps H_u; H is symmetric, so row i of this thread's result is written as
            // column i (consecutive lanes -> consecutive addresses)
            const int g = 2 * pr + u_out;
            if (g < nlist && i_row < D) {
                float *J = Jbuf + (size_t)g * D * D;
#pragma unroll
                for (int e = 0; e < 64; e++) {
                    const int j = j0 + e;
                    if (j < D) {
                        const float H = -acc[e] - (i_row == j ? inv_sp2 : 0.0f);
                        J[(size_t)j * D + i_row] = eps * H + (i_row == j ? 1.0f : 0.0f);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kIssWarp) tmem_dealloc(tm, kTmemCols);
    if (tid == 0 && *abort_f && timeout) atomicExch(timeout, 1u);
}

}  // namespace

bool hess_tc_supported(int D, int N) { return D > 64 && D <= kM && N > 0; }

size_t hess_tc_image_bytes(int N) { return (size_t)((N + kNB - 1) / kNB) * kChunk; }

cudaError_t launch_hess_tc_pack(const float *X, int N, int D, void *img, cudaStream_t st) {
    const int nch = (N + kNB - 1) / kNB;
    const int total = nch * kM * kNB;
    hess_tc_pack_kernel<<<(total + 255) / 256, 256, 0, st>>>(X, N, D, nch,
                                                            static_cast<unsigned char *>(img));
    return cudaGetLastError();
}

cudaError_t launch_hess_logreg_tc(int nlist, const int *list, int D, int N, const void *img,
                                  const float *s0, const float *s, float eps, float inv_sp2,
                                  float *Jbuf, unsigned int *timeout, unsigned int spin_limit,
                                  cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    cudaError_t e = ensure_dyn_smem(hess_logreg_tc_kernel, kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int npairs = (nlist + 1) / 2;
    const int grid = npairs < sms ? npairs : sms;
    hess_logreg_tc_kernel<<<grid, kThreads, kSmemBytes, st>>>(
        nlist, list, D, N, static_cast<const unsigned char *>(img), s0, s, eps, inv_sp2, Jbuf,
        timeout, spin_limit ? spin_limit : kDefaultSpinLimit);
    return cudaGetLastError();
}

}  // namespace pm
