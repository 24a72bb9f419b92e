// Host side of libpmcmc: context, workspace, the C ABI of include/pmcmc.h and the Newton loop
// of Algorithm 1 (on the device in a conditional CUDA graph, host-driven where graphs are not
// available, or over sliding windows as in Section 3.4).  Every arithmetic step runs in the
// kernels; this file only sizes buffers, launches, and reads back the per-iteration statistics
// (or, for the asynchronous solve, has a kernel write them to device memory).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "eval.h"
#include "seq.h"
#include "internal.h"
#include "solve.h"

using namespace pm;

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
static pmcmc_status fail(pmcmc_ctx *c, pmcmc_status st, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

#define PM_CUDA(c, call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((c), PMCMC_ECUDA, "%s failed: %s (%s:%d)", #call,                    \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

namespace pm {

pmcmc_status set_error(pmcmc_ctx *c, pmcmc_status st, const char *msg) {
    return fail(c, st, "%s", msg);
}

// ------------------------------------------------------------------------------------------
// workspace
// ------------------------------------------------------------------------------------------
pmcmc_status ws_reserve(pmcmc_ctx *c, size_t bytes) {
    if (bytes <= c->ws_bytes) return PMCMC_OK;
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&c->ws, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&c->ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PMCMC_ENOMEM, "workspace allocation of %zu bytes failed", bytes);
        }
        want = bytes;
    }
    c->ws_bytes = want;
    c->ws_generation++;
    return PMCMC_OK;
}

size_t Carve::take(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    return off;
}

static void stats_reset_host(EvalStats &s) {
    s.err = kOrdNegInf;
    s.rmax = 0x8000000000000000ull;  // +0.0
    s.min_margin = 0xfff0000000000000ull;  // +inf
    s.accepts = 0;
    s.resets = 0;
    s.dmax = 0x8000000000000000ull;
}

__global__ void stats_reset_kernel(EvalStats *s, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        s[i].err = kOrdNegInf;
        s[i].rmax = 0x8000000000000000ull;
        s[i].min_margin = 0xfff0000000000000ull;
        s[i].accepts = 0;
        s[i].resets = 0;
        s[i].dmax = 0x8000000000000000ull;
    }
}

__global__ void broadcast_rows_kernel(void *dst, const void *row, int T, int D, int esz) {
    size_t n = (size_t)T * D;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        int d = (int)(i % D);
        if (esz == 8)
            ((double *)dst)[i] = ((const double *)row)[d];
        else
            ((float *)dst)[i] = ((const float *)row)[d];
    }
}

// Zero-padded copy of the design matrix: Xp[n][k] = X[n][k] for n < N, k < D, else 0.
__global__ void pad_rows_kernel(void *dst, const void *src, int N, int D, int Npad, int DP,
                                int esz) {
    size_t n = (size_t)Npad * DP;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(i / DP), k = (int)(i % DP);
        bool in = r < N && k < D;
        if (esz == 8)
            ((double *)dst)[i] = in ? ((const double *)src)[(size_t)r * D + k] : 0.0;
        else
            ((float *)dst)[i] = in ? ((const float *)src)[(size_t)r * D + k] : 0.f;
    }
}

// all-finite check of a device array (sets *flag to 1 on a non-finite entry)
__global__ void finite_check_kernel(const void *p, size_t n, int esz, int *flag) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        double v = esz == 8 ? ((const double *)p)[i] : (double)((const float *)p)[i];
        if (!isfinite(v)) *flag = 1;
    }
}

static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 8));
}

cudaError_t pad_rows_launch(void *dst, const void *src, int N, int D, int Npad, int DP, int esz,
                            cudaStream_t st) {
    pad_rows_kernel<<<grid_for((size_t)Npad * DP), 256, 0, st>>>(dst, src, N, D, Npad, DP, esz);
    return cudaGetLastError();
}

}  // namespace pm

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

void pmcmc_options_default(pmcmc_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->sampler = PMCMC_MALA;
    o->step = 0.01;
    o->leapfrog_L = 0;
    o->jac = PMCMC_JAC_DIAG;
    o->precision = PMCMC_F32;
    o->atol = 1e-5;
    o->rtol = 0.0;
    o->max_iters = 0;
    o->damping = 1.0;
    o->clip = 0;
    o->gate_grad = 1;
    o->seed = 0;
    o->chain_id = 0;
    o->spin_limit = 0;
    o->engine = 0;
    o->seq_after = 0;
    o->window = 0;
}

pmcmc_status pmcmc_create(pmcmc_ctx **out, int device) {
    if (!out) return PMCMC_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return PMCMC_EINVAL;
    }
    pmcmc_ctx *c = new pmcmc_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return PMCMC_ECUDA;
    }
    if (cudaMalloc(&c->ctl, sizeof(CtlBlock)) != cudaSuccess ||
        cudaMallocHost(&c->host_ctl, sizeof(CtlBlock)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PMCMC_ENOMEM;
    }
    CtlBlock init;
    memset(&init, 0, sizeof(init));
    init.scan.epoch = 1;
    for (int i = 0; i < kMaxStats; i++) stats_reset_host(init.stats[i]);
    if (cudaMemcpy(c->ctl, &init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        cudaGetLastError();
        pmcmc_destroy(c);
        return PMCMC_ECUDA;
    }
    *out = c;
    return PMCMC_OK;
}

pmcmc_status pmcmc_destroy(pmcmc_ctx *c) {
    if (!c) return PMCMC_OK;
    cudaSetDevice(c->device);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->batch_graph_exec) cudaGraphExecDestroy(c->batch_graph_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t &q : c->seq_streams)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t &e : c->seq_events)
        if (e) cudaEventDestroy(e);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->ws) cudaFree(c->ws);
    if (c->aux) cudaFree(c->aux);
    if (c->seq_desc) cudaFree(c->seq_desc);
    if (c->ctl) cudaFree(c->ctl);
    if (c->host_ctl) cudaFreeHost(c->host_ctl);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (int i = 0; i < 6; i++)
        if (c->pev[i]) cudaEventDestroy(c->pev[i]);
    delete c;
    return PMCMC_OK;
}

const char *pmcmc_last_error(pmcmc_ctx *c) { return c ? c->err.c_str() : "null context"; }

pmcmc_status pmcmc_profile_enable(pmcmc_ctx *c, int enable) {
    if (!c) return PMCMC_EINVAL;
    PM_CUDA(c, cudaSetDevice(c->device));
    if (enable && !c->pev[0])
        for (int i = 0; i < 6; i++) PM_CUDA(c, cudaEventCreate(&c->pev[i]));
    c->prof_on = enable ? 1 : 0;
    if (enable) memset(&c->prof, 0, sizeof(c->prof));
    return PMCMC_OK;
}

pmcmc_status pmcmc_profile_get(pmcmc_ctx *c, pmcmc_profile *out) {
    if (!c || !out) return PMCMC_EINVAL;
    *out = c->prof;
    return PMCMC_OK;
}

pmcmc_status pmcmc_gen_noise(pmcmc_ctx *c, unsigned long long seed, unsigned int chain, int T,
                             int D, pmcmc_precision prec, void *xi, double *u, void *stream) {
    if (!c) return PMCMC_EINVAL;
    if (T < 0 || D < 0 || (T > 0 && D > 0 && !xi && !u))
        return fail(c, PMCMC_EINVAL, "gen_noise: invalid sizes or no output");
    if (T == 0) return PMCMC_OK;
    PM_CUDA(c, cudaSetDevice(c->device));
    PM_CUDA(c, launch_noise(seed, chain, T, D, prec == PMCMC_F64, D > 0 ? xi : nullptr, u,
                            (cudaStream_t)stream));
    return PMCMC_OK;
}

pmcmc_status pmcmc_scan(pmcmc_ctx *c, pmcmc_jac kind, pmcmc_precision prec, int T, int D,
                        const void *a, const void *b, void *s, void *stream) {
    if (!c) return PMCMC_EINVAL;
    if (T < 0 || D <= 0 || !a || !b || !s) return fail(c, PMCMC_EINVAL, "scan: invalid arguments");
    if (T == 0) return PMCMC_OK;
    PM_CUDA(c, cudaSetDevice(c->device));
    const bool f64 = prec == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    cudaStream_t st = (cudaStream_t)stream;
    ScanWork w;
    int tiles;
    int tile_t = 0;
    if (kind == PMCMC_JAC_DIAG) {
        if (D > 256) return fail(c, PMCMC_EUNSUPPORTED, "scan: diagonal scan supports D <= 256");
        tile_t = diag_scan_tile(T, D, rb);
        tiles = ceil_div(T, tile_t);
    } else if (kind == PMCMC_JAC_DENSE) {
        if (D > 32) return fail(c, PMCMC_EUNSUPPORTED, "scan: dense scan supports D <= 32");
        if (prec == PMCMC_F32_SCAN_BF16) {  // compositions on the tensor cores
            if (D <= 4) return fail(c, PMCMC_EUNSUPPORTED, "scan: bfloat16 dense scan needs D > 4");
            tile_t = dense_tc_chunk(T);
            tiles = ceil_div(T, 4 * tile_t);
        } else {
            tile_t = dense_scan_chunk(T, D);
            tiles = ceil_div(T, tile_t);
        }
    } else {
        return fail(c, PMCMC_EINVAL, "scan: kind must be DIAG or DENSE");
    }
    Carve cv;
    size_t o_flags = cv.take(sizeof(unsigned int) * tiles);
    size_t o_agg = cv.take((size_t)rb * tiles * ((size_t)D * D + 2 * D));
    size_t o_incl = cv.take((size_t)rb * tiles * D);
    pmcmc_status ps = ws_reserve(c, cv.used);
    if (ps != PMCMC_OK) return ps;
    char *base = (char *)c->ws;
    w.flags = (unsigned int *)(base + o_flags);
    w.agg = base + o_agg;
    w.incl = base + o_incl;
    w.max_tiles = tiles;
    w.ctl = &c->ctl->scan;
    if (c->flags_generation != c->ws_generation || c->flags_zeroed < (size_t)tiles) {
        PM_CUDA(c, cudaMemsetAsync(w.flags, 0, sizeof(unsigned int) * tiles, st));
    }
    // flags of this layout are zero or carry an older epoch from here on
    c->flags_generation = c->ws_generation;
    c->flags_zeroed = std::max(c->flags_zeroed, (size_t)tiles);
    c->flags_offset = o_flags;
    if (kind == PMCMC_JAC_DIAG)
        PM_CUDA(c, launch_scan_diag(f64, prec == PMCMC_F32_SCAN_BF16 ? 1 : 0, T, D, tile_t, a, b,
                                    s, nullptr, w, nullptr, nullptr, kDefaultSpinLimit, st));
    else if (prec == PMCMC_F32_SCAN_BF16)
        PM_CUDA(c, launch_scan_dense_tc(true, T, D, tile_t, a, b, s, nullptr, w, nullptr, nullptr,
                                        kDefaultSpinLimit, st));
    else
        PM_CUDA(c, launch_scan_dense(f64, T, D, tile_t, a, b, s, nullptr, w, nullptr, nullptr,
                                     kDefaultSpinLimit, st));
    return PMCMC_OK;
}

pmcmc_status pmcmc_scan_plan(pmcmc_jac kind, pmcmc_precision prec, int T, int D, int *kernel_out,
                             int *tile_out, int *tiles_out, int *max_tiles_out) {
    if (kind != PMCMC_JAC_DIAG) return PMCMC_EUNSUPPORTED;
    if (T <= 0 || D <= 0 || !kernel_out || !tile_out || !tiles_out || !max_tiles_out) return PMCMC_EINVAL;
    if (prec != PMCMC_F64 && prec != PMCMC_F32 && prec != PMCMC_F32_SCAN_BF16) return PMCMC_EINVAL;
    if (D > 256) return PMCMC_EUNSUPPORTED;
    const bool f64 = prec == PMCMC_F64;
    plan_scan_diag(f64, prec == PMCMC_F32_SCAN_BF16 ? 1 : 0, T, D, kernel_out, tile_out, tiles_out);
    // the look-back workspace pmcmc_scan reserves: one flag, aggregate and inclusive value per tile
    *max_tiles_out = ceil_div(T, diag_scan_tile(T, D, f64 ? 8 : 4));
    return PMCMC_OK;
}

}  // extern "C"

// ==========================================================================================
// Solve plumbing
// ==========================================================================================
namespace pm {

pmcmc_status check_problem(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                           const void *s0, bool sequential) {
    if (!tg || !o || !s0) return fail(c, PMCMC_EINVAL, "null target, options or s0");
    if (T < 0) return fail(c, PMCMC_EINVAL, "T must be >= 0");
    const int D = tg->D;
    if (D <= 0) return fail(c, PMCMC_EINVAL, "D must be > 0");
    if (o->sampler != PMCMC_MALA && o->sampler != PMCMC_HMC && o->sampler != PMCMC_HMC_PAR_LEAPFROG &&
        o->sampler != PMCMC_GIBBS)
        return fail(c, PMCMC_EINVAL, "unknown sampler");
    if (o->sampler != PMCMC_GIBBS && !(o->step > 0.0)) return fail(c, PMCMC_EINVAL, "step must be > 0");
    if ((o->sampler == PMCMC_GIBBS) != (tg->kind == PMCMC_SCHOOLS))
        return fail(c, PMCMC_EINVAL, "PMCMC_GIBBS runs on (only) the PMCMC_SCHOOLS target");
    if ((o->sampler == PMCMC_HMC || o->sampler == PMCMC_HMC_PAR_LEAPFROG) && o->leapfrog_L < 1)
        return fail(c, PMCMC_EINVAL, "HMC needs leapfrog_L >= 1");
    if (o->precision < PMCMC_F64 || o->precision > PMCMC_F32_SCAN_BF16)
        return fail(c, PMCMC_EINVAL, "unknown precision");
    if (o->jac < PMCMC_JAC_DENSE || o->jac > PMCMC_JAC_ZERO)
        return fail(c, PMCMC_EINVAL, "unknown Jacobian kind");
    switch (tg->kind) {
    case PMCMC_GAUSSIAN:
        if (!tg->mean || !tg->prec) return fail(c, PMCMC_EINVAL, "Gaussian needs mean and prec");
        if (D > 32) return fail(c, PMCMC_EUNSUPPORTED, "Gaussian target supports D <= 32");
        break;
    case PMCMC_BANANA:
        if (D != 2) return fail(c, PMCMC_EINVAL, "banana target has D = 2");
        break;
    case PMCMC_SCHOOLS:
        if (!tg->X || tg->N <= 0) return fail(c, PMCMC_EINVAL, "schools needs X (S x N scores), N > 0");
        if (!gibbs_supported(D, tg->N))
            return fail(c, PMCMC_EUNSUPPORTED, "schools target has D = 2 + 2 S with 1 <= S <= 15");
        if (tg->Q) return fail(c, PMCMC_EUNSUPPORTED, "no basis reparameterisation for Gibbs");
        if (o->jac != PMCMC_JAC_DENSE && o->jac != PMCMC_JAC_DIAG && o->jac != PMCMC_JAC_ZERO)
            return fail(c, PMCMC_EUNSUPPORTED, "Gibbs supports DENSE, DIAG and ZERO Jacobians");
        break;
    case PMCMC_LOGREG:
        if (!tg->X || !tg->y || tg->N <= 0) return fail(c, PMCMC_EINVAL, "logreg needs X, y, N > 0");
        if (!(tg->prior_scale > 0.0)) return fail(c, PMCMC_EINVAL, "prior_scale must be > 0");
        if (logreg_padded_dim(D) < 0) return fail(c, PMCMC_EUNSUPPORTED, "logreg supports D <= 128");
        if (o->precision == PMCMC_F64 && D > 64 && !sequential)  // the sequential loop takes D <= 128
            return fail(c, PMCMC_EUNSUPPORTED, "logreg in FP64 supports D <= 64");
        break;
    default:
        return fail(c, PMCMC_EINVAL, "unknown target kind");
    }
    if (o->jac == PMCMC_JAC_BLOCK2 && o->sampler != PMCMC_HMC_PAR_LEAPFROG)
        return fail(c, PMCMC_EINVAL, "BLOCK2 Jacobian is for PMCMC_HMC_PAR_LEAPFROG");
    if (o->jac == PMCMC_JAC_DENSE) {
        if (D > 32) return fail(c, PMCMC_EUNSUPPORTED, "dense Newton supports D <= 32");
        if (o->precision == PMCMC_F32_SCAN_BF16 && D <= 4)
            return fail(c, PMCMC_EUNSUPPORTED, "dense Newton with bfloat16 compositions needs D > 4");
        if (tg->kind == PMCMC_LOGREG && o->sampler != PMCMC_MALA)
            return fail(c, PMCMC_EUNSUPPORTED, "dense logreg Jacobian is for MALA");
    }
    if (tg->kind == PMCMC_LOGREG && o->sampler != PMCMC_MALA && !sequential)
        return fail(c, PMCMC_EUNSUPPORTED, "logreg Newton solves support MALA");
    return PMCMC_OK;
}

void fill_eval_args(EvalArgs &A, const pmcmc_target *tg, const pmcmc_options *o, int T) {
    A.target = tg->kind;
    A.sampler = o->sampler;
    A.T = T;
    A.D = tg->D;
    A.L = o->leapfrog_L;
    A.N = tg->N;
    A.eps = o->step;
    A.sigma_p = tg->prior_scale > 0 ? tg->prior_scale : 1.0;
    A.jac = o->jac;
    A.gate_grad = o->gate_grad;
    A.damping = o->damping > 0 ? o->damping : 1.0;
    A.clip = o->clip;
    A.rtol = o->rtol;
    A.f64 = o->precision == PMCMC_F64;
    A.bf16 = o->precision == PMCMC_F32_SCAN_BF16;
    A.mu = tg->mean;
    A.P = tg->prec;
    A.X = tg->X;
    A.y = tg->y;
    A.seed = o->seed;
    A.chain = o->chain_id;
    A.engine = o->engine;
}

// Whether the evaluate pass of this problem runs on the tensor-core kernel.
static bool uses_tc(const pmcmc_target *tg, const pmcmc_options *o, int T) {
    EvalArgs A;
    fill_eval_args(A, tg, o, T);
    return logreg_tc_supported(A);
}

// Whether the dense Jacobian of this problem is assembled on the tensor cores.
static bool uses_jac_tc(const pmcmc_target *tg, const pmcmc_options *o, int T) {
    EvalArgs A;
    fill_eval_args(A, tg, o, T);
    return logreg_jac_tc_supported(A);
}

// Workspace plan for one solve.
struct Plan {
    size_t o_a = 0, o_b = 0, o_xi = 0, o_u = 0, o_xp = 0, o_w = 0, o_ru = 0, o_rv = 0, o_acc = 0;
    size_t o_flags = 0, o_agg = 0, o_incl = 0, o_tmp = 0, o_img = 0, o_pimg = 0;
    bool tc = false, jtc = false;
    int tiles = 0, tile_t = 0;
    // Newton update fused into the tensor-core evaluate kernel: second iterate buffer, and flags
    // and aggregates of its 128-timestep tiles
    bool fused = false;
    int ftiles = 0;
    size_t o_salt = 0, o_fflags = 0, o_fagg = 0;
    size_t bytes = 0;
};

// The fused evaluate-and-update path: the tensor-core evaluate kernel in FP32 (the bfloat16
// pair variant keeps the separate scan, which is what stores the pairs in bfloat16).
// PMCMC_FUSED_UPDATE=0 selects the separate scan (measurements).
static bool fused_update(bool tc, const pmcmc_options *o) {
    if (!tc || o->precision != PMCMC_F32 || o->jac == PMCMC_JAC_DENSE) return false;
    const char *e = getenv("PMCMC_FUSED_UPDATE");
    return !(e && e[0] == '0');
}

static Plan make_plan(const pmcmc_target *tg, const pmcmc_options *o, int T, bool gen_noise,
                      bool need_tmp) {
    Plan p;
    Carve cv;
    const int D = tg->D;
    const bool f64 = o->precision == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    const int sb = o->precision == PMCMC_F32_SCAN_BF16 ? 2 : rb;
    const bool dense = o->jac == PMCMC_JAC_DENSE;
    p.o_a = cv.take(dense ? (size_t)rb * T * D * D : (size_t)sb * T * D);  // dense J in the arithmetic type
    p.o_b = cv.take((size_t)sb * T * D);
    if (gen_noise) {
        p.o_xi = cv.take((size_t)rb * T * D);
        p.o_u = cv.take(sizeof(double) * (size_t)T);
    }
    if (tg->kind == PMCMC_LOGREG) {
        const int DP = logreg_padded_dim(D);
        const int Npad = ceil_div(tg->N, 64) * 64;
        p.o_xp = cv.take((size_t)rb * Npad * DP);
        p.tc = uses_tc(tg, o, T);
        if (p.tc) p.o_img = cv.take(logreg_tc_image_bytes(tg->N));
        if (dense) {
            p.o_w = cv.take((size_t)rb * T * tg->N);
            p.o_ru = cv.take((size_t)rb * T * D);
            p.o_rv = cv.take((size_t)rb * T * D);
            p.jtc = uses_jac_tc(tg, o, T);
            if (p.jtc) p.o_pimg = cv.take(logreg_pair_image_bytes(tg->N, D));
        }
    }
    p.o_acc = cv.take((size_t)T);
    if (dense && o->precision == PMCMC_F32_SCAN_BF16) {  // tensor-core compositions, 4 chunks a tile
        p.tile_t = dense_tc_chunk(T);
        p.tiles = std::max(1, ceil_div(T, 4 * p.tile_t));
    } else {
        p.tile_t = dense ? dense_scan_chunk(T, D) : diag_scan_tile(T, D, rb);
        p.tiles = std::max(1, ceil_div(T, p.tile_t));
    }
    p.o_flags = cv.take(sizeof(unsigned int) * p.tiles);
    p.o_agg = cv.take((size_t)rb * p.tiles * ((size_t)D * D + 2 * D));
    p.o_incl = cv.take((size_t)rb * p.tiles * D);
    if (need_tmp) p.o_tmp = cv.take((size_t)rb * T * D);
    p.fused = fused_update(p.tc, o);
    if (p.fused) {
        p.ftiles = ceil_div(T, kTcTileT);
        p.o_salt = cv.take((size_t)rb * T * D);
        p.o_fflags = cv.take(sizeof(unsigned int) * (size_t)p.ftiles);
        p.o_fagg = cv.take(sizeof(float) * (size_t)p.ftiles * 64);
    }
    p.bytes = cv.used;
    return p;
}

}  // namespace pm

extern "C" pmcmc_status pmcmc_solve(pmcmc_ctx *c, const pmcmc_target *tg,
                                    const pmcmc_options *o, int T, const void *s0,
                                    const void *s_init, const void *xi, const double *u,
                                    void *s_out, pmcmc_result *res, void *stream) {
    if (!c) return PMCMC_EINVAL;
    if (res) memset(res, 0, sizeof(*res));
    pmcmc_status ps = check_problem(c, tg, o, T, s0, false);
    if (ps != PMCMC_OK) return ps;
    if (T > 0 && !s_out) return fail(c, PMCMC_EINVAL, "s_out is NULL");
    if ((xi == nullptr) != (u == nullptr)) return fail(c, PMCMC_EINVAL, "pass both xi and u, or neither");
    if (o->sampler == PMCMC_GIBBS && !xi)
        return fail(c, PMCMC_EINVAL, "Gibbs needs xi (its reparameterisation noise) and u");
    if (T == 0) {
        if (res) res->status = PMCMC_OK;
        return PMCMC_OK;
    }
    PM_CUDA(c, cudaSetDevice(c->device));
    if (tg->Q) return solve_with_basis(c, tg, o, T, s0, s_init, xi, u, s_out, res, stream);
    if (o->window > 0 && o->window < T) {
        if (tg->Q || o->sampler == PMCMC_HMC_PAR_LEAPFROG)
            return fail(c, PMCMC_EUNSUPPORTED, "sliding window: not with Q or HMC_PAR_LEAPFROG");
        return window_solve(c, tg, o, T, s0, s_init, xi, u, s_out, res, stream);
    }
    if (o->sampler == PMCMC_HMC_PAR_LEAPFROG)
        return solve_par_leapfrog(c, tg, o, T, s0, xi, u, s_out, res, stream);
    return newton_solve(c, tg, o, T, s0, s_init, xi, u, s_out, res, stream);
}

extern "C" pmcmc_status pmcmc_solve_async(pmcmc_ctx *c, const pmcmc_target *tg,
                                          const pmcmc_options *o, int T, const void *s0,
                                          const void *s_init, const void *xi, const double *u,
                                          void *s_out, pmcmc_result *res_dev, void *stream) {
    if (!c) return PMCMC_EINVAL;
    pmcmc_status ps = check_problem(c, tg, o, T, s0, false);
    if (ps != PMCMC_OK) return ps;
    if (!res_dev) return fail(c, PMCMC_EINVAL, "res_dev is NULL");
    if (T > 0 && !s_out) return fail(c, PMCMC_EINVAL, "s_out is NULL");
    if ((xi == nullptr) != (u == nullptr)) return fail(c, PMCMC_EINVAL, "pass both xi and u, or neither");
    if (o->sampler == PMCMC_GIBBS && !xi)
        return fail(c, PMCMC_EINVAL, "Gibbs needs xi (its reparameterisation noise) and u");
    if (tg->Q || o->sampler == PMCMC_HMC_PAR_LEAPFROG || (o->window > 0 && o->window < T))
        return fail(c, PMCMC_EUNSUPPORTED, "async solve: not with Q, HMC_PAR_LEAPFROG or a window");
    PM_CUDA(c, cudaSetDevice(c->device));
    if (T == 0) {  // all-zero result: status PMCMC_OK, no iterations
        PM_CUDA(c, cudaMemsetAsync(res_dev, 0, sizeof(pmcmc_result), (cudaStream_t)stream));
        return PMCMC_OK;
    }
    return newton_solve(c, tg, o, T, s0, s_init, xi, u, s_out, nullptr, stream, res_dev);
}

namespace pm {

// Device-side control of the Newton loop (Algorithm 1): decides convergence from the residual
// statistics of the evaluation just finished, keeps them for the host, and sets the WHILE
// condition of the graph (1: run the scan and another iteration; 0: stop).
__global__ void loop_ctl_kernel(CtlBlock *c, cudaGraphConditionalHandle h, double atol,
                                int max_iters) {
    loop_control_step(c, h, atol, max_iters);
}

// Fused update: the iterate of Newton iteration k lives in s_out for even k and in s_alt for
// odd k; after the loop the returned iterate is copied to s_out when it is in s_alt.
__global__ void select_result_kernel(const CtlBlock *c, float *__restrict__ s_out,
                                     const float *__restrict__ s_alt, size_t n) {
    if ((c->iter & 1) == 0) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s_out[i] = s_alt[i];
}

__global__ void loop_init_kernel(CtlBlock *c) {
    c->iter = 0;
    c->skip = 0;
    c->converged = 0;
    EvalStats &s = c->stats[0];
    s.err = kOrdNegInf;
    s.rmax = 0x8000000000000000ull;
    s.min_margin = 0xfff0000000000000ull;
    s.accepts = 0;
    s.resets = 0;
    s.dmax = 0x8000000000000000ull;
}

// Build (or reuse) the graph  [ WHILE { evaluate; control; scan } ]  for this solve.
static pmcmc_status build_loop_graph(pmcmc_ctx *c, const std::string &key, const pmcmc_target *tg,
                                     const pmcmc_options *o, const EvalArgs &A, const Plan &p,
                                     const ScanWork &w, void *s_out, const void *s0, int max_iters,
                                     unsigned int spin) {
    if (c->graph_exec && c->graph_key == key) return PMCMC_OK;
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_key.clear();
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return PMCMC_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return PMCMC_ECUDA;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t cs = c->cap_stream;
        ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const bool f64 = o->precision == PMCMC_F64;
            cudaError_t e = cudaSuccess;
            // fused path: the evaluate kernel's last tile also controls the loop
            EvalArgs Ag = A;
            if (p.fused) {
                Ag.loop = c->ctl;
                Ag.loop_handle = (unsigned long long)h;
                Ag.loop_atol = o->atol;
                Ag.loop_max_iters = max_iters;
            }
            if (tg->kind == PMCMC_LOGREG) {
                e = launch_eval_logreg(Ag, cs);
                if (e == cudaSuccess && o->jac == PMCMC_JAC_DENSE) e = launch_logreg_dense_jac(Ag, cs);
            } else {
                e = launch_eval_small(Ag, cs);
            }
            if (e == cudaSuccess && !p.fused) {
                loop_ctl_kernel<<<1, 1, 0, cs>>>(c->ctl, h, o->atol, max_iters);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && !p.fused) {  // the fused evaluate kernel applied the update
                if (o->jac == PMCMC_JAC_DENSE && A.bf16)
                    e = launch_scan_dense_tc(false, A.T, A.D, p.tile_t, A.a_out, A.b_out, s_out, s0, w,
                                             A.stats, &c->ctl->skip, spin, cs);
                else if (o->jac == PMCMC_JAC_DENSE)
                    e = launch_scan_dense(f64, A.T, A.D, p.tile_t, A.a_out, A.b_out, s_out, s0, w,
                                          A.stats, &c->ctl->skip, spin, cs);
                else
                    e = launch_scan_diag(f64, A.bf16 ? 1 : 0, A.T, A.D, p.tile_t, A.a_out, A.b_out,
                                         s_out, s0, w, A.stats, &c->ctl->skip, spin, cs);
            }
            cudaGraph_t out = nullptr;
            cudaError_t ce = cudaStreamEndCapture(cs, &out);
            ok = e == cudaSuccess && ce == cudaSuccess;
        }
    }
    cudaGraphExec_t ge = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return PMCMC_EUNSUPPORTED;
    }
    c->graph = g;
    c->graph_exec = ge;
    c->graph_key = key;
    return PMCMC_OK;
}

// The result of a device-side loop, written on the device (pmcmc_solve_async): the same fields
// the synchronous path reads back from the control block.
__global__ void write_result_kernel(CtlBlock *c, int T, pmcmc_result *r) {
    const bool timeout = c->scan.timeout != 0;
    r->status = c->nonfinite_input ? PMCMC_ENAN
                : timeout          ? PMCMC_ETIMEOUT
                : c->converged     ? PMCMC_OK
                                   : PMCMC_NOT_CONVERGED;
    if (timeout) c->scan.timeout = 0;
    r->iters = c->iter;
    r->max_residual = ord_decode(c->stats[1].rmax);
    r->accept_rate = (double)c->stats[1].accepts / (double)T;
    r->min_margin = ord_decode(c->stats[1].min_margin);
    r->nonfinite_resets = (int)c->stats[0].resets;
    r->elapsed_ms = 0.0f;
    r->sequential = 0;
}

pmcmc_status newton_solve(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                          const void *s0, const void *s_init, const void *xi, const double *u,
                          void *s_out, pmcmc_result *res, void *stream, pmcmc_result *res_dev) {
    cudaStream_t st = (cudaStream_t)stream;
    const int D = tg->D;
    const bool f64 = o->precision == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    const bool gen = xi == nullptr;
    Plan p = make_plan(tg, o, T, gen, false);
    pmcmc_status ps = ws_reserve(c, p.bytes);
    if (ps != PMCMC_OK) return ps;
    char *base = (char *)c->ws;
    ScanWork w;
    w.flags = (unsigned int *)(base + p.o_flags);
    w.agg = base + p.o_agg;
    w.incl = base + p.o_incl;
    w.max_tiles = p.tiles;
    w.ctl = &c->ctl->scan;
    if (c->flags_generation != c->ws_generation || c->flags_offset != p.o_flags ||
        c->flags_zeroed < (size_t)p.tiles) {
        PM_CUDA(c, cudaMemsetAsync(w.flags, 0, sizeof(unsigned int) * p.tiles, st));
        c->flags_generation = c->ws_generation;
        c->flags_offset = p.o_flags;
        c->flags_zeroed = p.tiles;
    }
    // the fused update's flags: this region may have held other data since its last use
    if (p.fused) PM_CUDA(c, cudaMemsetAsync(base + p.o_fflags, 0, sizeof(unsigned int) * p.ftiles, st));
    // inputs
    if (gen) {
        xi = base + p.o_xi;
        u = (const double *)(base + p.o_u);
        PM_CUDA(c, launch_noise(o->seed, o->chain_id, T, D, f64, (void *)xi, (double *)u, st));
        prof_count(c);
    }
    if (tg->kind == PMCMC_LOGREG) {
        const int DP = logreg_padded_dim(D);
        const int Npad = ceil_div(tg->N, 64) * 64;
        pad_rows_kernel<<<grid_for((size_t)Npad * DP), 256, 0, st>>>(base + p.o_xp, tg->X, tg->N,
                                                                     D, Npad, DP, rb);
        PM_CUDA(c, cudaGetLastError());
        prof_count(c);
        if (p.tc) {
            PM_CUDA(c, launch_logreg_tc_pack(tg->X, tg->y, tg->N, D, base + p.o_img, st));
            prof_count(c);
        }
        if (p.jtc) {
            PM_CUDA(c, launch_logreg_pair_pack(tg->X, tg->N, D, base + p.o_pimg, st));
            prof_count(c);
        }
    }
    // initial guess: s^(0) = s_init, or s0 broadcast (Appendix B)
    if (s_init) {
        if (s_init != s_out)
            PM_CUDA(c, cudaMemcpyAsync(s_out, s_init, (size_t)rb * T * D, cudaMemcpyDeviceToDevice, st));
    } else {
        broadcast_rows_kernel<<<grid_for((size_t)T * D), 256, 0, st>>>(s_out, s0, T, D, rb);
        PM_CUDA(c, cudaGetLastError());
        prof_count(c);
    }
    // finite check of s0 / the initial guess
    {
        int *flag = &c->ctl->nonfinite_input;
        PM_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), st));
        finite_check_kernel<<<grid_for((size_t)T * D), 256, 0, st>>>(s_out, (size_t)T * D, rb, flag);
        finite_check_kernel<<<1, 256, 0, st>>>(s0, (size_t)D, rb, flag);
        PM_CUDA(c, cudaGetLastError());
        prof_count(c, 2);
    }

    EvalArgs A;
    fill_eval_args(A, tg, o, T);
    A.s0 = s0;
    A.s = s_out;
    A.xi = xi;
    A.u = u;
    A.Xp = base + p.o_xp;
    A.a_out = base + p.o_a;
    A.b_out = base + p.o_b;
    A.acc_out = (unsigned char *)(base + p.o_acc);
    if (tg->kind == PMCMC_LOGREG && o->jac == PMCMC_JAC_DENSE) {
        A.w_out = base + p.o_w;
        A.rank1_u = base + p.o_ru;
        A.rank1_v = base + p.o_rv;
    }
    EvalStats *stats = &c->ctl->stats[0];
    A.stats = stats;
    A.iter = &c->ctl->iter;
    const int max_iters = o->max_iters > 0 ? o->max_iters : T;
    const unsigned int spin = o->spin_limit > 0 ? (unsigned int)o->spin_limit : kDefaultSpinLimit;
    if (p.tc) A.tc_img = base + p.o_img;
    if (p.jtc) A.pair_img = base + p.o_pimg;
    A.timeout = &c->ctl->scan.timeout;
    A.spin_limit = spin;
    if (p.fused) {
        A.a_out = nullptr;  // the pairs never leave the kernel
        A.b_out = nullptr;
        A.s_alt = base + p.o_salt;
        A.fs_flags = (unsigned int *)(base + p.o_fflags);
        A.fs_agg = (float *)(base + p.o_fagg);
        A.fs_ctl = &c->ctl->scan;
    }
    const double atol = o->atol;

    CtlBlock *h = c->host_ctl;
    if (!c->prof_on && !c->no_graph) {
        char kb[768];
        snprintf(kb, sizeof(kb),
                 "%llu|%d|%d|%d|%d|%d|%d|%d|%.17g|%.17g|%d|%.17g|%d|%d|%.17g|%.17g|%d|%u|%llu|%u|%d|%d|"
                 "%p|%p|%p|%p|%p|%p|%p|%p|%p",
                 c->ws_generation, T, D, tg->N, (int)tg->kind, (int)o->sampler, o->leapfrog_L,
                 (int)o->jac, o->step, tg->prior_scale, (int)o->precision, o->damping, o->clip,
                 o->gate_grad, o->atol, o->rtol, max_iters, spin, o->seed, o->chain_id, o->engine, (int)p.fused,
                 s0, s_out,
                 xi, (const void *)u, tg->mean, tg->prec, tg->X, tg->y, (void *)base);
        pmcmc_status gs = build_loop_graph(c, kb, tg, o, A, p, w, s_out, s0, max_iters, spin);
        if (gs == PMCMC_OK && res_dev) {  // enqueue only: the result lands in device memory
            loop_init_kernel<<<1, 1, 0, st>>>(c->ctl);
            PM_CUDA(c, cudaGetLastError());
            PM_CUDA(c, cudaGraphLaunch(c->graph_exec, st));
            if (p.fused) {
                select_result_kernel<<<grid_for((size_t)T * D), 256, 0, st>>>(
                    c->ctl, (float *)s_out, (const float *)(base + p.o_salt), (size_t)T * D);
                PM_CUDA(c, cudaGetLastError());
            }
            write_result_kernel<<<1, 1, 0, st>>>(c->ctl, T, res_dev);
            PM_CUDA(c, cudaGetLastError());
            return PMCMC_OK;
        }
        if (gs == PMCMC_OK) {
            PM_CUDA(c, cudaEventRecord(c->ev0, st));
            loop_init_kernel<<<1, 1, 0, st>>>(c->ctl);
            PM_CUDA(c, cudaGetLastError());
            PM_CUDA(c, cudaGraphLaunch(c->graph_exec, st));
            if (p.fused) {
                select_result_kernel<<<grid_for((size_t)T * D), 256, 0, st>>>(
                    c->ctl, (float *)s_out, (const float *)(base + p.o_salt), (size_t)T * D);
                PM_CUDA(c, cudaGetLastError());
            }
            PM_CUDA(c, cudaEventRecord(c->ev1, st));
            PM_CUDA(c, cudaMemcpyAsync(h, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st));
            PM_CUDA(c, cudaStreamSynchronize(st));
            float gms = 0.f;
            cudaEventElapsedTime(&gms, c->ev0, c->ev1);
            if (h->nonfinite_input) return fail(c, PMCMC_ENAN, "s0 or the initial guess is not finite");
            pmcmc_status status = h->converged ? PMCMC_OK : PMCMC_NOT_CONVERGED;
            if (h->scan.timeout) {
                unsigned int zero = 0;
                cudaMemcpy(&c->ctl->scan.timeout, &zero, sizeof(zero), cudaMemcpyHostToDevice);
                status = PMCMC_ETIMEOUT;
                fail(c, status, "a bounded wait (scan look-back or evaluate pipeline) ran out");
            }
            if (res) {
                res->iters = h->iter;
                res->status = status;
                res->max_residual = ord_decode(h->stats[1].rmax);
                res->accept_rate = (double)h->stats[1].accepts / (double)T;
                res->min_margin = ord_decode(h->stats[1].min_margin);
                res->nonfinite_resets = (int)h->stats[0].resets;
                res->elapsed_ms = gms;
            }
            return status;
        }
        c->no_graph = 1;  // conditional graphs refused: use the host-driven loop from now on
    }
    if (res_dev)
        return fail(c, PMCMC_EUNSUPPORTED, "async solve needs the device-side loop (conditional CUDA graphs, "
                                          "profiling off)");
    PM_CUDA(c, cudaEventRecord(c->ev0, st));
    int it = 0;
    bool converged = false;
    for (;;) {
        PM_CUDA(c, cudaMemcpyAsync(&c->ctl->iter, &it, sizeof(int), cudaMemcpyHostToDevice, st));
        stats_reset_kernel<<<1, 32, 0, st>>>(stats, 1);
        prof_count(c);
        prof_begin(c, 0, st);
        if (tg->kind == PMCMC_LOGREG) {
            PM_CUDA(c, launch_eval_logreg(A, st));
            prof_end(c, 0, st);
            prof_count(c);
            if (o->jac == PMCMC_JAC_DENSE) {
                prof_begin(c, 1, st);
                PM_CUDA(c, launch_logreg_dense_jac(A, st));
                prof_end(c, 1, st);
                prof_count(c);
            }
        } else {
            PM_CUDA(c, launch_eval_small(A, st));
            prof_end(c, 0, st);
            prof_count(c);
        }
        PM_CUDA(c, cudaMemcpyAsync(h, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st));
        PM_CUDA(c, cudaStreamSynchronize(st));
        prof_collect(c, 0);
        if (tg->kind == PMCMC_LOGREG && o->jac == PMCMC_JAC_DENSE) prof_collect(c, 1);
        if (h->nonfinite_input) return fail(c, PMCMC_ENAN, "s0 or the initial guess is not finite");
        const double err = ord_decode(h->stats[0].err);
        if (err <= atol) {
            converged = true;
            break;
        }
        if (it >= max_iters) break;
        if (p.fused) {  // the evaluate kernel wrote the next iterate to the other buffer
            it++;
            if (h->scan.timeout) break;
            continue;
        }
        prof_begin(c, 2, st);
        if (o->jac == PMCMC_JAC_DENSE && A.bf16)
            PM_CUDA(c, launch_scan_dense_tc(false, T, D, p.tile_t, A.a_out, A.b_out, s_out, s0, w, stats,
                                            nullptr, spin, st));
        else if (o->jac == PMCMC_JAC_DENSE)
            PM_CUDA(c, launch_scan_dense(f64, T, D, p.tile_t, A.a_out, A.b_out, s_out, s0, w, stats,
                                         nullptr, spin, st));
        else
            PM_CUDA(c, launch_scan_diag(f64, A.bf16 ? 1 : 0, T, D, p.tile_t, A.a_out, A.b_out, s_out,
                                        s0, w, stats, nullptr, spin, st));
        prof_end(c, 2, st);
        prof_count(c);
        it++;
        PM_CUDA(c, cudaMemcpyAsync(h, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st));
        PM_CUDA(c, cudaStreamSynchronize(st));
        prof_collect(c, 2);
        c->resets_accum += h->stats[0].resets;
        if (h->scan.timeout) break;
    }
    if (p.fused && (it & 1))
        PM_CUDA(c, cudaMemcpyAsync(s_out, base + p.o_salt, (size_t)rb * T * D, cudaMemcpyDeviceToDevice, st));
    PM_CUDA(c, cudaEventRecord(c->ev1, st));
    PM_CUDA(c, cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    pmcmc_status status = converged ? PMCMC_OK : PMCMC_NOT_CONVERGED;
    if (h->scan.timeout) {
        unsigned int zero = 0;
        cudaMemcpy(&c->ctl->scan.timeout, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        status = PMCMC_ETIMEOUT;
        fail(c, status, "a bounded wait (scan look-back or evaluate pipeline) ran out");
    }
    if (res) {
        res->iters = it;
        res->status = status;
        res->max_residual = ord_decode(h->stats[0].rmax);
        res->accept_rate = (double)h->stats[0].accepts / (double)T;
        res->min_margin = ord_decode(h->stats[0].min_margin);
        res->nonfinite_resets = (int)c->resets_accum;
        res->elapsed_ms = ms;
    }
    c->resets_accum = 0;
    return status;
}

// ------------------------------------------------------------------------------------------
// Sliding-window Newton updates (Section 3.4): each iteration evaluates f_t and J_t on the W
// steps from t0, the first step whose residual is not yet within tolerance, moves t0 past the
// converged prefix of the window, and applies the Newton update to the rest of the window with
// the carry zero at the new t0 (its predecessor is converged and is never changed again).  The
// first step after t0 is exact after one update, so t0 advances every iteration.
// ------------------------------------------------------------------------------------------
template <typename R, typename S_>
__global__ void first_unconverged_kernel(int n, int D, const S_ *__restrict__ r,
                                         const R *__restrict__ s, double atol, double rtol,
                                         int *first) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= (size_t)n * D) return;
    const double rv = fabs((double)load_as<S_, R>(r + e)), sv = fabs((double)s[e]);
    const double v = rv - rtol * sv;
    if (!(v <= atol)) atomicMin(first, (int)(e / D));  // NaN counts as not converged
}

// accepted steps among the window's first *first steps (the prefix that becomes frozen)
__global__ void window_accepts_kernel(const unsigned char *acc, const int *first, int *count) {
    int local = 0;
    const int k = *first;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) local += acc[t];
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

__global__ void set_int_kernel(int *p, int v) { *p = v; }

pmcmc_status window_solve(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                          const void *s0, const void *s_init, const void *xi, const double *u,
                          void *s_out, pmcmc_result *res, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int D = tg->D;
    const bool f64 = o->precision == PMCMC_F64;
    const bool bf16 = o->precision == PMCMC_F32_SCAN_BF16;
    const int rb = f64 ? 8 : 4;
    const int W = o->window;
    const bool gen = xi == nullptr;
    if (o->jac == PMCMC_JAC_DENSE && bf16)
        return fail(c, PMCMC_EUNSUPPORTED, "window: dense Newton in FP32 or FP64 (no bfloat16 compositions)");
    Plan p = make_plan(tg, o, W, false, false);
    Carve cv;
    cv.used = p.bytes;
    const size_t o_xi = gen ? cv.take((size_t)rb * T * D) : 0;
    const size_t o_u = gen ? cv.take(sizeof(double) * (size_t)T) : 0;
    pmcmc_status ps = ws_reserve(c, cv.used);
    if (ps != PMCMC_OK) return ps;
    char *base = (char *)c->ws;
    ScanWork w;
    w.flags = (unsigned int *)(base + p.o_flags);
    w.agg = base + p.o_agg;
    w.incl = base + p.o_incl;
    w.max_tiles = p.tiles;
    w.ctl = &c->ctl->scan;
    PM_CUDA(c, cudaMemsetAsync(w.flags, 0, sizeof(unsigned int) * p.tiles, st));
    c->flags_generation = ~0ull;  // the next whole-chain solve re-zeroes its flag area
    if (gen) {
        xi = base + o_xi;
        u = (const double *)(base + o_u);
        PM_CUDA(c, launch_noise(o->seed, o->chain_id, T, D, f64, (void *)xi, (double *)u, st));
    }
    if (tg->kind == PMCMC_LOGREG) {
        const int DP = logreg_padded_dim(D);
        const int Npad = ceil_div(tg->N, 64) * 64;
        pad_rows_kernel<<<grid_for((size_t)Npad * DP), 256, 0, st>>>(base + p.o_xp, tg->X, tg->N,
                                                                     D, Npad, DP, rb);
        PM_CUDA(c, cudaGetLastError());
        if (p.tc) PM_CUDA(c, launch_logreg_tc_pack(tg->X, tg->y, tg->N, D, base + p.o_img, st));
        if (p.jtc) PM_CUDA(c, launch_logreg_pair_pack(tg->X, tg->N, D, base + p.o_pimg, st));
    }
    if (s_init) {
        if (s_init != s_out)
            PM_CUDA(c, cudaMemcpyAsync(s_out, s_init, (size_t)rb * T * D, cudaMemcpyDeviceToDevice, st));
    } else {
        broadcast_rows_kernel<<<grid_for((size_t)T * D), 256, 0, st>>>(s_out, s0, T, D, rb);
        PM_CUDA(c, cudaGetLastError());
    }
    {
        int *flag = &c->ctl->nonfinite_input;
        PM_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), st));
        finite_check_kernel<<<grid_for((size_t)T * D), 256, 0, st>>>(s_out, (size_t)T * D, rb, flag);
        finite_check_kernel<<<1, 256, 0, st>>>(s0, (size_t)D, rb, flag);
        PM_CUDA(c, cudaGetLastError());
    }
    EvalArgs A;
    fill_eval_args(A, tg, o, W);
    A.Xp = base + p.o_xp;
    A.a_out = base + p.o_a;
    A.b_out = base + p.o_b;
    A.acc_out = (unsigned char *)(base + p.o_acc);
    if (tg->kind == PMCMC_LOGREG && o->jac == PMCMC_JAC_DENSE) {
        A.w_out = base + p.o_w;
        A.rank1_u = base + p.o_ru;
        A.rank1_v = base + p.o_rv;
    }
    EvalStats *stats = &c->ctl->stats[0];
    A.stats = stats;
    A.iter = &c->ctl->iter;
    const unsigned int spin = o->spin_limit > 0 ? (unsigned int)o->spin_limit : kDefaultSpinLimit;
    if (p.tc) A.tc_img = base + p.o_img;
    if (p.jtc) A.pair_img = base + p.o_pimg;
    A.timeout = &c->ctl->scan.timeout;
    A.spin_limit = spin;
    const int max_iters = o->max_iters > 0 ? o->max_iters : T;
    const size_t jrow = o->jac == PMCMC_JAC_DENSE ? (size_t)D * D : (size_t)D;
    const int sb = bf16 ? 2 : rb;
    CtlBlock *h = c->host_ctl;
    int *first = &c->ctl->first_bad, *wacc = &c->ctl->win_accepts;
    PM_CUDA(c, cudaMemsetAsync(wacc, 0, sizeof(int), st));
    PM_CUDA(c, cudaEventRecord(c->ev0, st));
    int it = 0, t0 = 0;
    bool converged = false;
    double rmax = 0.0, margin = INFINITY;
    for (;;) {
        const int n = std::min(W, T - t0);
        A.T = n;
        A.s0 = t0 == 0 ? s0 : (const char *)s_out + (size_t)rb * (t0 - 1) * D;
        A.s = (char *)s_out + (size_t)rb * t0 * D;
        A.xi = (const char *)xi + (size_t)rb * t0 * D;
        A.u = u + t0;
        PM_CUDA(c, cudaMemcpyAsync(&c->ctl->iter, &it, sizeof(int), cudaMemcpyHostToDevice, st));
        stats_reset_kernel<<<1, 32, 0, st>>>(stats, 1);
        if (tg->kind == PMCMC_LOGREG) {
            PM_CUDA(c, launch_eval_logreg(A, st));
            if (o->jac == PMCMC_JAC_DENSE) PM_CUDA(c, launch_logreg_dense_jac(A, st));
        } else {
            PM_CUDA(c, launch_eval_small(A, st));
        }
        set_int_kernel<<<1, 1, 0, st>>>(first, n);
        const size_t ne = (size_t)n * D;
        if (f64)
            first_unconverged_kernel<double, double><<<grid_for(ne), 256, 0, st>>>(
                n, D, (const double *)A.b_out, (const double *)A.s, o->atol, o->rtol, first);
        else if (bf16)
            first_unconverged_kernel<float, __nv_bfloat16><<<grid_for(ne), 256, 0, st>>>(
                n, D, (const __nv_bfloat16 *)A.b_out, (const float *)A.s, o->atol, o->rtol, first);
        else
            first_unconverged_kernel<float, float><<<grid_for(ne), 256, 0, st>>>(
                n, D, (const float *)A.b_out, (const float *)A.s, o->atol, o->rtol, first);
        window_accepts_kernel<<<std::max(1, std::min(64, ceil_div(n, 256))), 256, 0, st>>>(A.acc_out, first, wacc);
        PM_CUDA(c, cudaGetLastError());
        PM_CUDA(c, cudaMemcpyAsync(h, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st));
        PM_CUDA(c, cudaStreamSynchronize(st));
        if (h->nonfinite_input) return fail(c, PMCMC_ENAN, "s0 or the initial guess is not finite");
        rmax = std::max(rmax, ord_decode(h->stats[0].rmax));
        margin = std::min(margin, ord_decode(h->stats[0].min_margin));
        const int k = h->first_bad;
        if (t0 + k >= T) {
            converged = true;
            break;
        }
        if (k == n) {  // the whole window is converged: move on without an update
            t0 += k;
            continue;
        }
        if (it >= max_iters) break;
        // update the unconverged rest of the window, [t0 + k, t0 + n), with the carry zero at t0 + k
        const void *a = (const char *)A.a_out + (size_t)(o->jac == PMCMC_JAC_DENSE ? rb : sb) * k * jrow;
        const void *b = (const char *)A.b_out + (size_t)sb * k * D;
        void *sw = (char *)s_out + (size_t)rb * (t0 + k) * D;
        if (o->jac == PMCMC_JAC_DENSE)
            PM_CUDA(c, launch_scan_dense(f64, n - k, D, p.tile_t, a, b, sw, s0, w, stats, nullptr, spin, st));
        else
            PM_CUDA(c, launch_scan_diag(f64, bf16 ? 1 : 0, n - k, D, p.tile_t, a, b, sw, s0, w, stats,
                                        nullptr, spin, st));
        it++;
        t0 += k;
        PM_CUDA(c, cudaMemcpyAsync(h, c->ctl, sizeof(CtlBlock), cudaMemcpyDeviceToHost, st));
        PM_CUDA(c, cudaStreamSynchronize(st));
        c->resets_accum += h->stats[0].resets;
        if (h->scan.timeout) break;
    }
    PM_CUDA(c, cudaEventRecord(c->ev1, st));
    PM_CUDA(c, cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    pmcmc_status status = converged ? PMCMC_OK : PMCMC_NOT_CONVERGED;
    if (h->scan.timeout) {
        unsigned int zero = 0;
        cudaMemcpy(&c->ctl->scan.timeout, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        status = PMCMC_ETIMEOUT;
        fail(c, status, "a bounded wait (scan look-back or evaluate pipeline) ran out");
    }
    if (res) {
        res->iters = it;
        res->status = status;
        res->max_residual = rmax;
        res->accept_rate = (double)h->win_accepts / (double)T;
        res->min_margin = margin;
        res->nonfinite_resets = (int)c->resets_accum;
        res->elapsed_ms = ms;
    }
    c->resets_accum = 0;
    return status;
}

}  // namespace pm

extern "C" pmcmc_status pmcmc_linearize(pmcmc_ctx *c, const pmcmc_target *tg,
                                        const pmcmc_options *o, int T, const void *s0,
                                        const void *s, const void *xi, const double *u,
                                        void *f_out, void *jac_out, unsigned char *acc_out,
                                        double *ell_out, void *stream) {
    if (!c) return PMCMC_EINVAL;
    pmcmc_status ps = check_problem(c, tg, o, T, s0, false);
    if (ps != PMCMC_OK) return ps;
    if (o->sampler == PMCMC_HMC_PAR_LEAPFROG)
        return fail(c, PMCMC_EINVAL, "linearize: use MALA or HMC");
    if (!s || !xi || !u) return fail(c, PMCMC_EINVAL, "linearize needs s, xi and u");
    if (o->precision == PMCMC_F32_SCAN_BF16)
        return fail(c, PMCMC_EINVAL, "linearize: use F32 or F64");
    if (T == 0) return PMCMC_OK;
    PM_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int D = tg->D;
    const bool f64 = o->precision == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    Carve cv;
    size_t o_xp = 0, o_w = 0, o_ru = 0, o_rv = 0, o_acc = 0, o_j = 0, o_img = 0, o_pimg = 0;
    const bool dense = o->jac == PMCMC_JAC_DENSE;
    const bool tc = uses_tc(tg, o, T);
    const bool jtc = tg->kind == PMCMC_LOGREG && dense && uses_jac_tc(tg, o, T);
    if (tg->kind == PMCMC_LOGREG) {
        const int DP = logreg_padded_dim(D);
        o_xp = cv.take((size_t)rb * ceil_div(tg->N, 64) * 64 * DP);
        if (tc) o_img = cv.take(logreg_tc_image_bytes(tg->N));
        if (dense) {
            o_w = cv.take((size_t)rb * T * tg->N);
            o_ru = cv.take((size_t)rb * T * D);
            o_rv = cv.take((size_t)rb * T * D);
            o_acc = cv.take((size_t)T);
            if (jtc) o_pimg = cv.take(logreg_pair_image_bytes(tg->N, D));
        }
    }
    if (dense && !jac_out) o_j = cv.take((size_t)rb * T * D * D);
    ps = ws_reserve(c, std::max<size_t>(cv.used, 256));
    if (ps != PMCMC_OK) return ps;
    char *base = (char *)c->ws;
    EvalArgs A;
    fill_eval_args(A, tg, o, T);
    A.s0 = s0;
    A.s = s;
    A.xi = xi;
    A.u = u;
    A.f_out = f_out;
    A.a_out = jac_out ? jac_out : (dense ? (void *)(base + o_j) : nullptr);
    A.acc_out = acc_out;
    A.ell_out = ell_out;
    A.iter = nullptr;  // Hutchinson probes of Newton iteration 0, whatever ran before
    if (tg->kind == PMCMC_LOGREG) {
        const int DP = logreg_padded_dim(D);
        const int Npad = ceil_div(tg->N, 64) * 64;
        A.Xp = base + o_xp;
        pad_rows_kernel<<<grid_for((size_t)Npad * DP), 256, 0, st>>>(base + o_xp, tg->X, tg->N, D,
                                                                     Npad, DP, rb);
        if (tc) {
            PM_CUDA(c, launch_logreg_tc_pack(tg->X, tg->y, tg->N, D, base + o_img, st));
            A.tc_img = base + o_img;
            A.timeout = &c->ctl->scan.timeout;
            A.spin_limit = o->spin_limit > 0 ? (unsigned int)o->spin_limit : kDefaultSpinLimit;
        }
        if (dense) {
            A.w_out = base + o_w;
            A.rank1_u = base + o_ru;
            A.rank1_v = base + o_rv;
            if (!acc_out) A.acc_out = (unsigned char *)(base + o_acc);
            if (jtc) {
                PM_CUDA(c, launch_logreg_pair_pack(tg->X, tg->N, D, base + o_pimg, st));
                A.pair_img = base + o_pimg;
                A.timeout = &c->ctl->scan.timeout;
                A.spin_limit = o->spin_limit > 0 ? (unsigned int)o->spin_limit : kDefaultSpinLimit;
            }
        }
        PM_CUDA(c, launch_eval_logreg(A, st));
        if (dense) PM_CUDA(c, launch_logreg_dense_jac(A, st));
    } else {
        PM_CUDA(c, launch_eval_small(A, st));
    }
    PM_CUDA(c, cudaStreamSynchronize(st));
    if (tc || jtc) {
        unsigned int to = 0;
        PM_CUDA(c, cudaMemcpy(&to, &c->ctl->scan.timeout, sizeof(to), cudaMemcpyDeviceToHost));
        if (to) {
            const unsigned int zero = 0;
            cudaMemcpy(&c->ctl->scan.timeout, &zero, sizeof(zero), cudaMemcpyHostToDevice);
            return fail(c, PMCMC_ETIMEOUT, "a bounded wait of the evaluate pipeline ran out");
        }
    }
    return PMCMC_OK;
}

extern "C" pmcmc_status pmcmc_seq_solve(pmcmc_ctx *c, const pmcmc_target *tg,
                                        const pmcmc_options *o, int T, const void *s0,
                                        const void *xi, const double *u, void *s_out,
                                        unsigned char *accept_out, void *stream) {
    if (!c) return PMCMC_EINVAL;
    pmcmc_status ps = check_problem(c, tg, o, T, s0, true);
    if (ps != PMCMC_OK) return ps;
    if (!s_out || !xi || !u) return fail(c, PMCMC_EINVAL, "seq_solve needs xi, u and s_out");
    if (o->precision == PMCMC_F32_SCAN_BF16) return fail(c, PMCMC_EINVAL, "seq_solve: F32 or F64");
    if (T == 0) return PMCMC_OK;
    PM_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    pmcmc_options oo = *o;
    if (oo.sampler == PMCMC_HMC_PAR_LEAPFROG) oo.sampler = PMCMC_HMC;
    EvalArgs A;
    fill_eval_args(A, tg, &oo, T);
    A.s0 = s0;
    A.xi = xi;
    A.u = u;
    A.f_out = s_out;
    A.acc_out = accept_out;
    if (tg->kind == PMCMC_LOGREG) {
        if (tg->N > 20000) return fail(c, PMCMC_EUNSUPPORTED, "seq_solve logreg supports N <= 20000");
        PM_CUDA(c, launch_seq_logreg(A, st));
    } else if (tg->kind == PMCMC_GAUSSIAN && tg->D >= 4 && seq_fast_supported(seq_chain_from(A))) {
        // one CTA: the D x D products spread over D threads (a lone thread serves D < 4)
        PM_CUDA(c, launch_seq_chain(seq_chain_from(A), A.f64, st));
    } else {
        PM_CUDA(c, launch_seq_small(A, st));
    }
    return PMCMC_OK;
}
