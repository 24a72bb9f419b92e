// pmcmc_scan_noalloc: the diagonal look-back scan without any allocation.
//
// Some callers cannot allocate device memory: code that runs while a CUDA stream is being
// captured into a graph (cudaMalloc is not a stream operation and breaks or is forbidden during
// capture), real-time or embedded hosts that fix their memory budget at start-up, and plugins
// living inside a framework whose own allocator owns the device (a stray cudaMalloc there
// fragments its pool or fails under its memory cap).  They cannot create a context either,
// because a context owns a workspace.  This entry point takes no context: the look-back flags,
// tile aggregates and control words live in one file-scope device array of fixed size, which
// every GPU that loads the library holds until the process exits.
//
// Set-up: the first call on each device (with that device current) resolves the array's device
// address with cudaGetSymbolAddress; make that first call before any stream capture.  The
// address is cached per device ordinal for the life of the process, so it assumes the device's
// primary context (the runtime API's) and no cudaDeviceReset in between.  Each call
// then clears the parts that must start at zero (the tile flags of this call and the ticket,
// done and timeout words) with cudaMemsetAsync on the caller's stream, and launches the same
// scan kernel pmcmc_scan uses.  All calls share the array and each overwrites what the previous
// one left, so calls whose executions overlap on the GPU (different streams without ordering)
// race and give wrong results; order them on one stream.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace pm {
namespace {

constexpr size_t kNoallocScratchBytes = 8u << 20;  // 8 MiB per device

// One control block followed by the flag / aggregate / inclusive areas of one scan.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

}  // namespace
}  // namespace pm

extern "C" pmcmc_status pmcmc_scan_noalloc(pmcmc_precision prec, int T, int D, const void *a,
                                           const void *b, void *s, void *stream) {
    using namespace pm;
    if (T < 0 || D <= 0 || !a || !b || !s) return PMCMC_EINVAL;
    if (prec != PMCMC_F64 && prec != PMCMC_F32 && prec != PMCMC_F32_SCAN_BF16) return PMCMC_EINVAL;
    if (D > 256) return PMCMC_EUNSUPPORTED;
    if (T == 0) return PMCMC_OK;
    const bool f64 = prec == PMCMC_F64;
    const int rb = f64 ? 8 : 4;
    const int tile_t = diag_scan_tile(T, D, rb);
    const int tiles = ceil_div(T, tile_t);
    // layout inside the array: [ScanCtl | flags | aggregates | inclusive], 256-byte aligned
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_flags = up(sizeof(ScanCtl));
    const size_t o_agg = up(o_flags + sizeof(unsigned int) * (size_t)tiles);
    const size_t o_incl = up(o_agg + (size_t)rb * tiles * 2 * D);
    const size_t need = o_incl + (size_t)rb * tiles * D;
    if (need > kNoallocScratchBytes) return PMCMC_EUNSUPPORTED;  // beyond the static maximum

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PMCMC_ECUDA;
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return PMCMC_ECUDA;
            }
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    char *p = (char *)base;
    ScanCtl *ctl = (ScanCtl *)p;
    // ticket, done and timeout start at zero; the epoch word is left as the last call set it
    if (cudaMemsetAsync(&ctl->ticket, 0, 2 * sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(&ctl->timeout, 0, sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(p + o_flags, 0, sizeof(unsigned int) * (size_t)tiles, st) != cudaSuccess) {
        cudaGetLastError();
        return PMCMC_ECUDA;
    }
    ScanWork w;
    w.flags = (unsigned int *)(p + o_flags);
    w.agg = p + o_agg;
    w.incl = p + o_incl;
    w.max_tiles = tiles;
    w.ctl = ctl;
    cudaError_t e = launch_scan_diag(f64, prec == PMCMC_F32_SCAN_BF16 ? 1 : 0, T, D, tile_t, a, b, s,
                                     nullptr, w, nullptr, nullptr, kDefaultSpinLimit, st);
    if (e == cudaErrorInvalidValue) {  // a kernel's own tile-count guard refused the size
        cudaGetLastError();
        return PMCMC_EUNSUPPORTED;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PMCMC_ECUDA;
    }
    return PMCMC_OK;
}
