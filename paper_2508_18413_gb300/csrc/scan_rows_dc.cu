// The row kernel of the diagonal scan with D a compile-time constant (D = 1, 2, 4, 8, 16, 32;
// 8 rows per warp): the channel-segmented shuffle offsets, lane roles and element indices fold
// into constants.  A translation unit of its own so that the library builds in parallel.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "scan_rows.cuh"

namespace pm {

namespace {

// CTAs of `kernel` (256 threads) resident on the device at once, cached per kernel.
template <class K>
int resident(K kernel) {
    static const void *keys[32] = {};
    static int vals[32] = {};
    static int n = 0;
    const void *key = reinterpret_cast<const void *>(kernel);
    for (int i = 0; i < n; i++)
        if (keys[i] == key) return vals[i];
    int per_sm = 1, dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (n < 32) {
        keys[n] = key;
        vals[n++] = per_sm * sms;
    }
    return per_sm * sms;
}

template <typename R, typename S, int DC>
cudaError_t run(int T, int nsub, const void *a, const void *b, void *s, const void *s_reset,
                const ScanWork &w, EvalStats *stats, const int *skip, unsigned int spin, cudaStream_t st) {
    const int ntiles = ceil_div(T, 8 * 8 * nsub * (32 / DC));
    if (ntiles > w.max_tiles) return cudaErrorInvalidValue;
    auto k = scan_diag_rows_kernel<R, S, 8, DC>;
    prefer_shared(k);
    k<<<std::min(ntiles, resident(k)), 256, 0, st>>>(T, DC, nsub, (const S *)a, (const S *)b, (R *)s,
                                                    (const R *)s_reset, w.flags, (R *)w.agg, (R *)w.incl,
                                                    w.ctl, stats, skip, spin);
    return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t run_d(int T, int D, int nsub, const void *a, const void *b, void *s, const void *s_reset,
                  const ScanWork &w, EvalStats *stats, const int *skip, unsigned int spin, cudaStream_t st) {
    switch (D) {
        case 1: return run<R, S, 1>(T, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
        case 2: return run<R, S, 2>(T, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
        case 4: return run<R, S, 4>(T, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
        case 8: return run<R, S, 8>(T, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
        case 16: return run<R, S, 16>(T, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
        case 32: return run<R, S, 32>(T, nsub, a, b, s, s_reset, w, stats, skip, spin, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_scan_rows_dconst(int kind, int T, int D, int nsub, const void *a, const void *b, void *s,
                                    const void *s_reset, const ScanWork &w, EvalStats *stats,
                                    const int *skip, unsigned int spin_limit, cudaStream_t st) {
    if (kind == 2) return run_d<double, double>(T, D, nsub, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    if (kind == 1)
        return run_d<float, __nv_bfloat16>(T, D, nsub, a, b, s, s_reset, w, stats, skip, spin_limit, st);
    return run_d<float, float>(T, D, nsub, a, b, s, s_reset, w, stats, skip, spin_limit, st);
}

}  // namespace pm
