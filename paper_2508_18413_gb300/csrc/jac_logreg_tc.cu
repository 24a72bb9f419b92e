// Dense Jacobian of MALA on Bayesian logistic regression (DEER, Eq. 2; the MALA map of
// Section 3.2 with its derivative through the proposal), D <= 32, FP32, on the tensor cores:
//   J_t = g_t (I + eps H_t) + (1 - g_t) I + u_t v_t^T,   H_t = -X^T W_t X - I / sp^2,
// with W_t = diag(sigmoid'(z_tn)), z_t = X s_{t-1}, and the accept indicator g_t and the gate
// vectors u_t, v_t written by the evaluate pass.  The entries of X^T W_t X over the pairs
// (i <= j) are, for a tile of 128 timesteps, one GEMM against a pair image of the design:
//   S[t, p] = sum_n w_tn Y_np,   Y_np = X_ni X_nj,
// with M = 128 timesteps (one TMEM lane each), N = the pairs of this CTA's group (up to 512
// columns in MMA blocks of up to 256: the P = D (D + 1) / 2 pairs are split over ceil(P / 512)
// CTAs, one for D <= 31), K = the data rows in
// chunks of 32 (tcgen05.mma kind::tf32, one product per term).  One tf32 product suffices:
// J only shapes the Newton step (any J leads to the same fixed point), and 2^-11 relative per
// term keeps J within 1e-3 of its FP32 value.
//
// Roles (160 threads): warps 0-3 stage the A operand (their 32 rows of w for each chunk, tf32
// values in the 128-byte-swizzled K-major layout) and, at the end, read the accumulator lanes
// and write J; lane 0 of warp 4 streams the pair-image chunks with bulk copies and issues the
// MMAs.  Two stages.  Every wait is bounded: a wait that runs out raises the CTA's abort flag,
// the roles stop, in-flight copies and MMAs are drained, TMEM is freed and the launch's
// timeout word is set.
#include "common.cuh"
#include "eval.h"
#include "internal.h"
#include "tc.cuh"

namespace pm {
namespace {

using namespace tc;

constexpr int kM = 128;                       // timesteps per tile
constexpr int kNB = 32;                       // data rows per chunk (K)
// pairs per CTA at most: two MMA column blocks of up to 256 (one 512-column TMEM allocation),
// so one CTA takes all pairs of a tile for D <= 31 and the grid is one wave of tiles
constexpr int kGroupCols = 512;
constexpr int kMmaCols = 256;                 // MMA N per column block
constexpr int kThreads = 160;
constexpr int kIss = 4;                       // issuer warp
constexpr int kAOp = kM * kNB * 4;            // A stage: 128 x 32 floats = 16 KB
constexpr int kBOp = kGroupCols * kNB * 4;    // B stage: up to 512 x 32 floats = 64 KB
constexpr int kStages = 2;
constexpr int oA = 0;
constexpr int oB = kStages * kAOp;
constexpr int oBar = oB + kStages * kBOp;
constexpr int bFull = 0, bAready = bFull + kStages, bEmpty = bAready + kStages, bDone = bEmpty + kStages,
              kNumBars = bDone + 1;
constexpr int oMisc = oBar + 8 * kNumBars;    // tmem address, abort flag
constexpr int oPairs = oMisc + 16;            // uint8 pairs (i, j) of this group: 2 x 256
constexpr int oOwn = oPairs + 2 * kGroupCols; // uint8 per entry of J_t: 1 if its pair is in this group
constexpr int kSmemUsed = oOwn + 32 * 32;
// J staging after the products: the operand stages are free then, 24 KB per epilogue warp,
// slices of kSlice entries x 32 timesteps (row stride 33 words)
constexpr int kWarpStage = (kStages * (kAOp + kBOp)) / 4 / 4;  // floats per warp
constexpr int kSlice = kWarpStage / 33;
constexpr int kSmemBytes = kSmemUsed + 1024;  // + alignment slack
constexpr unsigned int kDrain = 1u << 20;
static_assert(oB % 1024 == 0 && kAOp % 1024 == 0 && kBOp % 1024 == 0, "operand alignment");

__host__ __device__ constexpr int npairs(int D) { return D * (D + 1) / 2; }
__host__ __device__ constexpr int ngroups(int D) { return (npairs(D) + kGroupCols - 1) / kGroupCols; }
// MMA N of group g (a multiple of 16) and the byte stride of one chunk block of the image
__host__ __device__ constexpr int group_cols(int D, int g) {
    return ((((g + 1) * kGroupCols < npairs(D) ? kGroupCols : npairs(D) - g * kGroupCols) + 15) / 16) * 16;
}

__device__ __forceinline__ float post_jac(float v, float damping, int clip) {
    v *= damping;
    if (clip) v = fminf(fmaxf(v, -1.0f), 1.0f);
    return v;
}

// Pair image: block (g, k) holds the group's pairs p (rows, padded to a multiple of 16) times
// the 32 data rows of chunk k (K), Y_np = X_ni X_nj rounded to tf32, 128-byte swizzled.
__global__ void pair_pack_kernel(const float *__restrict__ X, int N, int D, unsigned char *__restrict__ img) {
    const int k = blockIdx.x, g = blockIdx.y;
    const int P = npairs(D), ncol = group_cols(D, g);
    unsigned char *blk = img + ((size_t)g * gridDim.x + k) * kBOp;
    for (int e = threadIdx.x; e < ncol * kNB; e += blockDim.x) {
        const int pl = e / kNB, nl = e % kNB;
        const int p = g * kGroupCols + pl, n = k * kNB + nl;
        float v = 0.0f;
        if (p < P && n < N) {
            int i = 0, rem = p;  // p -> (i, j), row-major over i <= j
            while (rem >= D - i) {
                rem -= D - i;
                i++;
            }
            const int j = i + rem;
            v = X[(size_t)n * D + i] * X[(size_t)n * D + j];
        }
        *reinterpret_cast<float *>(blk + swz128((uint32_t)pl, (uint32_t)nl)) = to_tf32(v);
    }
}

__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort, unsigned int limit) {
    const bool ok = mbar_wait(bar, parity, abort, limit);
    return __all_sync(0xffffffffu, ok);
}

__global__ void __launch_bounds__(kThreads, 1) jac_logreg_tc_kernel(EvalArgs A) {
    if (A.skip && *(volatile const int *)A.skip) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const uint32_t sb = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = A.T, D = A.D, N = A.N, DD = D * D;
    const int g = blockIdx.y, t0 = blockIdx.x * kM;
    const int P = npairs(D), ncol = group_cols(D, g);
    const int nch = (N + kNB - 1) / kNB;
    const unsigned int limit = A.spin_limit ? A.spin_limit : kDefaultSpinLimit;
    volatile int *abort_f = reinterpret_cast<volatile int *>(sm + oMisc + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + oMisc);
    unsigned char *pij = sm + oPairs;  // [0, kGroupCols): i, [kGroupCols, 2 kGroupCols): j
    unsigned char *own = sm + oOwn;
    auto bar = [&](int i) -> uint32_t { return sb + oBar + 8u * (uint32_t)i; };
    const uint32_t tcols = ncol <= 32 ? 32u : ncol <= 64 ? 64u : ncol <= 128 ? 128u : ncol <= 256 ? 256u : 512u;

    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(bar(bFull + s), 1);
            mbar_init(bar(bAready + s), 4);
            mbar_init(bar(bEmpty + s), 1);
        }
        mbar_init(bar(bDone), 1);
        *abort_f = 0;
        fence_barrier_init();
    }
    if (tid < D) {  // the group's pair table
        const int base = tid * D - tid * (tid - 1) / 2;
        for (int j = tid; j < D; j++) {
            const int pl = base + (j - tid) - g * kGroupCols;
            if (pl >= 0 && pl < kGroupCols) {
                pij[pl] = (unsigned char)tid;
                pij[kGroupCols + pl] = (unsigned char)j;
            }
        }
    }
    for (int e = tid; e < DD; e += kThreads) {
        const int a = e / D, b = e - a * D;
        const int i = min(a, b), j = max(a, b);
        const int pl = i * D - i * (i - 1) / 2 + (j - i) - g * kGroupCols;
        own[e] = (pl >= 0 && pl < kGroupCols) ? 1 : 0;
    }
    if (warp == kIss) {
        tmem_alloc(smem_u32(tmem_slot), tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tmem_slot;
    const unsigned char *img = static_cast<const unsigned char *>(A.pair_img) + (size_t)g * nch * kBOp;
    const uint32_t bbytes = (uint32_t)ncol * kNB * 4u;

    if (warp == kIss) {
        if (lane == 0) {
            // column blocks: [0, 256) and [256, ncol), each a multiple of 16
            const int nblk = ncol > kMmaCols ? 2 : 1;
            const uint32_t idesc0 = idesc_tf32(kM, ncol > kMmaCols ? kMmaCols : ncol);
            const uint32_t idesc1 = idesc_tf32(kM, ncol > kMmaCols ? ncol - kMmaCols : 16);
            int ncopy = 0, nmma = 0;
            bool ok = true;
            auto copy = [&](int k) {
                const int s = k % kStages;
                mbar_arrive_expect_tx(bar(bFull + s), bbytes);
                bulk_g2s(sb + oB + s * kBOp, img + (size_t)k * kBOp, bbytes, bar(bFull + s));
                ncopy++;
            };
            for (int k = 0; k < kStages && k < nch; k++) copy(k);
            for (int k = 0; k < nch && ok; k++) {
                const int s = k % kStages;
                const uint32_t par = (uint32_t)(k / kStages) & 1u;
                if (!(ok = mbar_wait(bar(bFull + s), par, abort_f, limit))) break;
                if (!(ok = mbar_wait(bar(bAready + s), par, abort_f, limit))) break;
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < kNB / 8; kk++) {
                    const uint64_t ad = sdesc(sb + oA + s * kAOp + 32 * kk);
                    mma_tf32(tm, ad, sdesc(sb + oB + s * kBOp + 32 * kk), idesc0, (k > 0 || kk > 0) ? 1u : 0u);
                    if (nblk > 1)  // rows 256.. of the B stage: 256 rows x 128 bytes further on
                        mma_tf32(tm + (uint32_t)kMmaCols, ad, sdesc(sb + oB + s * kBOp + kMmaCols * 128 + 32 * kk),
                                 idesc1, (k > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(bar(bEmpty + s));
                nmma++;
                if (k + kStages < nch) {  // this stage's MMAs read B: wait for them before the refill
                    if (!(ok = mbar_wait(bar(bEmpty + s), par, abort_f, limit))) break;
                    copy(k + kStages);
                }
            }
            mma_commit(bar(bDone));
            // drain: every issued copy has landed, every issued MMA has completed
            mbar_wait_drain(bar(bDone), 0, kDrain);
            for (int q = ncopy > kStages ? ncopy - kStages : 0; q < ncopy; q++)
                mbar_wait_drain(bar(bFull + q % kStages), (uint32_t)(q / kStages) & 1u, kDrain);
            (void)nmma;
        }
        __syncwarp();
    } else {
        // ---------------- A operand: 32 rows of w per warp per chunk ----------------
        const int t = t0 + warp * 32 + lane;  // this lane's timestep in the epilogue
        const bool tv = t < T;
        // The warp's 32 rows of a chunk are read row by row, lane = column (one 128-byte request
        // per row); lane c holds column c of every row and writes it into the swizzled operand.
        const int rw0 = t0 + warp * 32;  // first timestep of the warp's rows
        const float *wbase = static_cast<const float *>(A.w_out);
        bool ok = true;
        float wv[32];
        const int nrows = min(32, T - rw0);  // valid rows of the warp (warp-uniform)
        auto load_w = [&](int k) {
            const int n = k * kNB + lane;
            const bool nv = n < N;
            const float *p = wbase + (size_t)(rw0 < T ? rw0 : 0) * N + (nv ? n : 0);
#pragma unroll
            for (int q = 0; q < 32; q++) {
                wv[q] = (q < nrows && nv) ? __ldg(p) : 0.0f;
                p += N;
            }
        };
        load_w(0);
        for (int k = 0; k < nch; k++) {
            const int s = k % kStages;
            if (k >= kStages && !(ok = warp_wait(bar(bEmpty + s), (uint32_t)((k - kStages) / kStages) & 1u, abort_f, limit)))
                break;
            unsigned char *as = sm + oA + s * kAOp;
#pragma unroll
            for (int q = 0; q < 32; q++)
                *reinterpret_cast<float *>(as + swz128((uint32_t)(warp * 32 + q), (uint32_t)lane)) = wv[q];
            fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(bAready + s));
            if (k + 1 < nch) load_w(k + 1);
        }
        // ---------------- J_t from the accumulator lanes ----------------
        if (ok) ok = warp_wait(bar(bDone), 0u, abort_f, limit);
        tc_fence_after();
        // J_t of the warp's 32 timesteps, in slices of kSlice entries: each lane computes its
        // entries of the slice from the accumulator columns into shared memory (entry-major,
        // one column per lane), then the warp writes the slice row by row, consecutive lanes
        // on consecutive entries of one J_t, only the entries whose pair is in this group.
        // `ok` is uniform across the warp, `tv` is not (a ragged last tile): every lane takes
        // part in the warp-collective TMEM loads.
        if (ok) {
            const float eps = (float)A.eps, damping = (float)A.damping;
            const float inv_sp2 = (float)(1.0 / (A.sigma_p * A.sigma_p));
            const float ga = (tv && A.acc_out[t]) ? 1.0f : 0.0f;
            const float *ru = static_cast<const float *>(A.rank1_u) + (size_t)(tv ? t : 0) * D;
            const float *rv = static_cast<const float *>(A.rank1_v) + (size_t)(tv ? t : 0) * D;
            float *Jw = static_cast<float *>(A.a_out) + (size_t)(t0 + warp * 32) * DD;
            float *stg = reinterpret_cast<float *>(sm + oA) + warp * kWarpStage;
            const uint32_t lrow = tm + ((uint32_t)(warp * 32) << 16);
            const int nt = min(32, T - (t0 + warp * 32));  // valid timesteps of this warp
            for (int e0 = 0; e0 < DD && nt > 0; e0 += kSlice) {
                const int e1 = min(e0 + kSlice, DD);
                for (int cb = 0; cb < ncol; cb += 16) {
                    float v[16];
                    tmem_ld16(lrow + (uint32_t)cb, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 16; c++) {
                        const int pl = cb + c;
                        if (g * kGroupCols + pl >= P) break;
                        const int i = pij[pl], j = pij[kGroupCols + pl];
                        const int eij = i * D + j, eji = j * D + i;
                        const bool in1 = eij >= e0 && eij < e1, in2 = i != j && eji >= e0 && eji < e1;
                        if (!(in1 || in2)) continue;
                        const float h = -v[c] - (i == j ? inv_sp2 : 0.0f);
                        const float base = ga * eps * h + (i == j ? 1.0f : 0.0f);
                        // the gate term u_t v_t^T is zero with the gate held (its vectors are
                        // then not written)
                        const float gij = A.gate_grad ? ru[i] * rv[j] : 0.0f;
                        const float gji = A.gate_grad ? ru[j] * rv[i] : 0.0f;
                        if (in1) stg[(eij - e0) * 33 + lane] = post_jac(base + gij, damping, A.clip);
                        if (in2) stg[(eji - e0) * 33 + lane] = post_jac(base + gji, damping, A.clip);
                    }
                }
                __syncwarp();
                for (int l = 0; l < nt; l++) {
                    float *Jt = Jw + (size_t)l * DD;
                    for (int e = e0 + lane; e < e1; e += 32)
                        if (own[e]) Jt[e] = stg[(e - e0) * 33 + l];
                }
                __syncwarp();
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kIss) {
        tc_fence_after();
        tmem_dealloc(tm, tcols);
    }
    if (*abort_f && tid == 0 && A.timeout) atomicExch(A.timeout, 1u);
}

}  // namespace

bool logreg_jac_tc_supported(const EvalArgs &A) {
    return !A.f64 && A.engine == 0 && A.target == PMCMC_LOGREG && A.sampler == PMCMC_MALA &&
           A.jac == PMCMC_JAC_DENSE && A.D >= 1 && A.D <= 32 && A.N >= 1;
}

size_t logreg_pair_image_bytes(int N, int D) {
    return (size_t)ngroups(D) * (size_t)ceil_div(N, kNB) * kBOp;
}

cudaError_t launch_logreg_pair_pack(const void *X, int N, int D, void *img, cudaStream_t st) {
    if (D < 1 || D > 32 || N < 1) return cudaErrorInvalidValue;
    pair_pack_kernel<<<dim3(ceil_div(N, kNB), ngroups(D)), 256, 0, st>>>(static_cast<const float *>(X), N, D,
                                                                        static_cast<unsigned char *>(img));
    return cudaGetLastError();
}

cudaError_t launch_jac_logreg_tc(const EvalArgs &A, cudaStream_t st) {
    if (!A.pair_img || reinterpret_cast<uintptr_t>(A.pair_img) % 16 != 0 || !A.w_out || !A.a_out ||
        !A.acc_out || (A.gate_grad && (!A.rank1_u || !A.rank1_v)))
        return cudaErrorInvalidValue;
    if (A.T <= 0) return cudaSuccess;
    cudaError_t e = ensure_dyn_smem(jac_logreg_tc_kernel, kSmemBytes);
    if (e != cudaSuccess) return e;
    jac_logreg_tc_kernel<<<dim3(ceil_div(A.T, kM), ngroups(A.D)), kThreads, kSmemBytes, st>>>(A);
    return cudaGetLastError();
}

}  // namespace pm
