// Dense Jacobians of held-decision MALA steps on the logistic target, on the tensor cores.
//
// For the adjoint (the reverse recursion of the fixed point with the decisions held), every
// accepted step t needs J_t = I + eps H(x_t) with x_t = s_{t-1} and
//   H(x) = -X^T diag(w) X - I / sigma_p^2,   w_n = sigmoid(z_n) (1 - sigmoid(z_n)),   z = X x,
// an N x D x D contraction per step: the dominant work of the adjoint (Section 3.2's MALA
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
constexpr int kWBytes = 2 * kNB * 4;      // w of the chunk's 32 rows for both steps
constexpr int kStageStride = 33 * 1024;  // image chunk + w, 1024-aligned
constexpr int kPeriod = 4;               // chunks per TMEM accumulator before it is drained
constexpr int kWorkWarps = 16, kWorkThreads = 32 * kWorkWarps;
constexpr int kIssWarp = kWorkWarps, kCopyWarp = kWorkWarps + 1;
constexpr int kThreads = 32 * (kWorkWarps + 2);
constexpr uint32_t kIdesc = idesc_tf32(kM, 2 * kM);
constexpr uint32_t kTmemCols = 512;      // two accumulators of 256 columns
constexpr unsigned int kDrainLimit = 1u << 20;

// shared-memory map (offsets from a 1024-aligned base)
constexpr int oStage = 0;
constexpr int oB = oStage + kStages * kStageStride;  // B hi (256 rows), then B lo
constexpr int bFull = 0, bEmpty = kStages, bBready = 2 * kStages, bBfree = bBready + 2,
              bAccFull = bBfree + 2, bAccEmpty = bAccFull + 2, bFin = bAccEmpty + 2,
              kNumBars = bFin + 1;
constexpr int oBar = oB + 4 * kTile;
constexpr int oMisc = oBar + 8 * kNumBars;        // tmem address, abort flag
constexpr int kSmemUsed = oMisc + 16;
constexpr int kSmemBytes = kSmemUsed + 1024;      // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(oB % 1024 == 0 && kStageStride % 1024 == 0 && kChunk + kWBytes <= kStageStride &&
                  oBar % 8 == 0,
              "alignment");

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

// W[g][n] = sigmoid'(X[n] . x_g) for the listed steps g (x_g = s_{list[g] - 1}, s0 for step 0)
// and n < ldw (zero for n >= N): a 64-step x 64-row tile per CTA, features in slices of 32
// through shared memory, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) hess_w_kernel(int nlist, const int *__restrict__ list, int D,
                                                     int N, int ldw, const float *__restrict__ X,
                                                     const float *__restrict__ s0,
                                                     const float *__restrict__ s, float *__restrict__ W) {
    __shared__ float xs[64][33], xr[64][33];
    const int g0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float acc[4][4] = {};
    for (int d0 = 0; d0 < D; d0 += 32) {
        __syncthreads();
        for (int e = tid; e < 64 * 32; e += 256) {
            const int r = e >> 5, d = d0 + (e & 31);
            const int g = g0 + r, n = n0 + r;
            float v = 0.0f;
            if (g < nlist && d < D) {
                const int t = list[g];
                v = t == 0 ? s0[d] : s[(size_t)(t - 1) * D + d];
            }
            xs[r][e & 31] = v;
            xr[r][e & 31] = (n < N && d < D) ? X[(size_t)n * D + d] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int d = 0; d < 32; d++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                a[i] = xs[4 * ty + i][d];
                b[i] = xr[4 * tx + i][d];
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int g = g0 + 4 * ty + i;
        const int n = n0 + 4 * tx;
        if (g >= nlist || n >= ldw) continue;
        float w4[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float sg = 1.0f / (1.0f + expf(-acc[i][j]));
            w4[j] = n + j < N ? sg * (1.0f - sg) : 0.0f;
        }
        *reinterpret_cast<float4 *>(W + (size_t)g * ldw + n) = make_float4(w4[0], w4[1], w4[2], w4[3]);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
hess_logreg_tc_kernel(int nlist, int D, int N, const unsigned char *__restrict__ img,
                      const float *__restrict__ W, int ldw, float eps, float inv_sp2,
                      float *__restrict__ Jbuf, unsigned int *timeout, unsigned int limit) {
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
                    const uint32_t dst = sb + oStage + st * kStageStride;
                    const int g0 = 2 * pr, g1 = 2 * pr + 1 < nlist ? 2 * pr + 1 : 2 * pr;
                    mbar_arrive_expect_tx(bar(bFull + st), kChunk + kWBytes);
                    bulk_g2s(dst, img + (size_t)c * kChunk, kChunk, bar(bFull + st));
                    bulk_g2s(dst + kChunk, W + (size_t)g0 * ldw + (size_t)c * kNB, kWBytes / 2, bar(bFull + st));
                    bulk_g2s(dst + kChunk + kWBytes / 2, W + (size_t)g1 * ldw + (size_t)c * kNB, kWBytes / 2,
                             bar(bFull + st));
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
                    const uint32_t a0 = sb + oStage + st * kStageStride;
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
        // Named barriers among the worker warps are never skipped by a subset of them: the
        // chunk loop has none, a failed wait only marks the warp's status, and the and-barrier
        // at the end of each pair makes the status common before the workers leave together.
        // B positions of this thread (fixed for every chunk): lane -> (row, chunk) so that each
        // quarter-warp covers two rows whose swizzled chunks fill all 32 banks (rows 8g + q and
        // 8g + q + 4, chunk lane % 4 of the half); two positions per half, rows < 128 -> step 0
        const int f_row0 = 8 * (tid >> 5) + ((lane >> 3) + 4 * ((lane >> 2) & 1));
        const int f_row1 = f_row0 + 8 * (kWorkThreads >> 5);
        const int f_u0 = f_row0 >> 7, f_u1 = f_row1 >> 7;
        const uint32_t f_off0 = swz128((uint32_t)(f_row0 & (kM - 1)), (uint32_t)(4 * (lane & 3)));
        const uint32_t f_off1 = swz128((uint32_t)(f_row1 & (kM - 1)), (uint32_t)(4 * (lane & 3)));
        int k = 0, gp = 0;
        for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
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
                for (int b8 = 0; b8 < 8; b8++) {
                    float v[8];
                    tmem_ld8(a + 8u * b8, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; e++) acc[8 * b8 + e] += v[e];
                }
                warp_arrive(bar(bAccEmpty + (p & 1)));
                return true;
            };
            for (int c = 0; c < nch; c++, k++) {
                const int st = k % kStages;
                const unsigned char *stg = sm + oStage + st * kStageStride;
                if (good) good = warp_wait(bar(bFull + st), (uint32_t)(k / kStages) & 1u, abort_f, limit);
                const float *wc = reinterpret_cast<const float *>(stg + kChunk);  // w of both steps
                // B = w (.) X^T for both steps; half h = K-steps 2h, 2h + 1 (16-byte chunks 4h..4h+3)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    if (good && k >= 1) good = warp_wait(bar(bBfree + h), (uint32_t)(k - 1) & 1u, abort_f, limit);
                    if (!good) continue;
#pragma unroll 1
                    for (int rep = 0; rep < 2; rep++) {
                        // half h uses the chunk 4 further along: swizzled offset bit 6 flips
                        const uint32_t off = (rep ? f_off1 : f_off0) ^ ((uint32_t)h << 6);
                        const int u = rep ? f_u1 : f_u0;
                        const float4 xh = *reinterpret_cast<const float4 *>(stg + off);
                        const float4 xl = *reinterpret_cast<const float4 *>(stg + kTile + off);
                        const float4 w4 = *reinterpret_cast<const float4 *>(wc + u * kNB + 16 * h + 4 * (lane & 3));
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
            if (good) good = drain(gp + nper - 1);
            gp += nper;
            if (!named_bar_and(1, kWorkThreads, good)) break;
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

size_t hess_tc_w_floats(int nlist, int N) { return (size_t)nlist * (size_t)((N + kNB - 1) / kNB * kNB); }

size_t hess_tc_image_bytes(int N) { return (size_t)((N + kNB - 1) / kNB) * kChunk; }

cudaError_t launch_hess_tc_pack(const float *X, int N, int D, void *img, cudaStream_t st) {
    const int nch = (N + kNB - 1) / kNB;
    const int total = nch * kM * kNB;
    hess_tc_pack_kernel<<<(total + 255) / 256, 256, 0, st>>>(X, N, D, nch,
                                                            static_cast<unsigned char *>(img));
    return cudaGetLastError();
}

cudaError_t launch_hess_logreg_tc(int nlist, const int *list, int D, int N, const float *X,
                                  const void *img, const float *s0, const float *s, float *W,
                                  float eps, float inv_sp2, float *Jbuf, unsigned int *timeout,
                                  unsigned int spin_limit, cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    const int ldw = (N + kNB - 1) / kNB * kNB;
    hess_w_kernel<<<dim3((ldw + 63) / 64, (nlist + 63) / 64), 256, 0, st>>>(nlist, list, D, N, ldw, X,
                                                                           s0, s, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = ensure_dyn_smem(hess_logreg_tc_kernel, kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int npairs = (nlist + 1) / 2;
    const int grid = npairs < sms ? npairs : sms;
    hess_logreg_tc_kernel<<<grid, kThreads, kSmemBytes, st>>>(
        nlist, D, N, static_cast<const unsigned char *>(img), W, ldw, eps, inv_sp2, Jbuf, timeout,
        spin_limit ? spin_limit : kDefaultSpinLimit);
    return cudaGetLastError();
}

}  // namespace pm
