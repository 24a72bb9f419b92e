// Shared device helpers for the parallel-Newton MCMC kernels (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pmcmc.h"

namespace pm {

constexpr int kWarp = 32;

// ------------------------------------------------------------------------------------------
// Storage <-> arithmetic conversion.  The scan may keep its affine pairs in bfloat16 while the
// arithmetic is FP32; all other buffers store the arithmetic type itself.
// ------------------------------------------------------------------------------------------
template <typename S, typename R>
__device__ __forceinline__ R load_as(const S *p) { return static_cast<R>(*p); }
template <>
__device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}
// read-only (non-coherent) load of data that no thread of the kernel writes
template <typename S, typename R>
__device__ __forceinline__ R ldg_as(const S *p) { return static_cast<R>(__ldg(p)); }
template <>
__device__ __forceinline__ float ldg_as<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <typename S, typename R>
__device__ __forceinline__ void store_as(S *p, R v) { *p = static_cast<S>(v); }
template <>
__device__ __forceinline__ void store_as<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}

template <typename R>
__device__ __forceinline__ bool finite(R v) { return isfinite(v); }

// ------------------------------------------------------------------------------------------
// Order-preserving double <-> uint64 encoding so max-reductions can use integer atomics.
// NaN is mapped to +inf (a non-finite value must never look converged).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ord_encode(double v) {
    if (isnan(v)) v = __longlong_as_double(0x7ff0000000000000ll);
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_decode(unsigned long long b) {
    unsigned long long r = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
    double d;
    memcpy(&d, &r, sizeof(d));
    return d;
}
constexpr unsigned long long kOrdNegInf = 0x000fffffffffffffull;  // ord_encode(-inf)

__device__ __forceinline__ void atomic_max_d(unsigned long long *addr, double v) {
    atomicMax(addr, ord_encode(v));
}
__device__ __forceinline__ void atomic_min_d(unsigned long long *addr, double v) {
    atomicMin(addr, ord_encode(v));
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------------------------------
// Acquire / release accesses for the decoupled look-back flags (GPU scope).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------------------------------------
// Per-launch device control block.  One lives in the context's workspace for each concurrent
// solve.  Tickets give tiles in dispatch order (forward progress of the look-back); the last
// CTA to finish resets them and advances `epoch`, which tags the look-back flags, so repeated
// launches (including graph replays) need no memset.
// ------------------------------------------------------------------------------------------
struct ScanCtl {
    unsigned int ticket;
    unsigned int done;
    unsigned int epoch;
    unsigned int timeout;  // set when a bounded look-back wait ran out
};

// Statistics of one evaluate-and-linearise pass.
struct EvalStats {
    unsigned long long err;        // ord-encoded max_{t,d} (|r| - rtol |s|)
    unsigned long long rmax;       // ord-encoded max |r|
    unsigned long long min_margin; // ord-encoded min_t |log alpha - log u|
    unsigned long long accepts;    // number of accepted steps
    unsigned long long resets;     // non-finite elements reset by the scan
    unsigned long long dmax;       // ord-encoded max |delta| of the last scan
};

__host__ __device__ inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// (k + 1/2) 2^-53 from the top 53 bits of the 64-bit word (hi:lo)
__device__ __forceinline__ double uniform53(unsigned int lo, unsigned int hi) {
    unsigned long long k = ((((unsigned long long)hi) << 32) | lo) >> 11;
    return ((double)k + 0.5) * (1.0 / 9007199254740992.0);
}

// Bounded spin helper: returns false once `limit` polls have elapsed.
struct Spin {
    unsigned int n = 0, limit;
    __device__ explicit Spin(unsigned int lim) : limit(lim) {}
    __device__ bool again() {
        if (++n >= limit) return false;
        if (n > 64) __nanosleep(n > 1024 ? 1000 : 64);
        return true;
    }
};

// Ask for the largest shared-memory carveout once per kernel: for kernels with little static
// shared memory the driver may otherwise pick an 8 KB configuration that admits one block per SM.
// Keyed by the kernel's address: kernels of identical signature share a template instance.
template <class K>
inline void prefer_shared(K kernel) {
    static const void *done[32] = {};
    static int n = 0;
    const void *key = reinterpret_cast<const void *>(kernel);
    for (int i = 0; i < n; i++)
        if (done[i] == key) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    if (n < 32) done[n++] = key;
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (cached per kernel).  Static
// plus dynamic shared memory above 48 KB needs this opt-in, so it is applied to every size.
template <class K>
inline cudaError_t ensure_dyn_smem(K kernel, size_t bytes) {
    static const void *keys[32] = {};
    static size_t vals[32] = {};
    static int n = 0;
    const void *key = reinterpret_cast<const void *>(kernel);
    int i = 0;
    for (; i < n; i++)
        if (keys[i] == key) break;
    if (i < n && vals[i] >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (i < n) {
        vals[i] = bytes;
    } else if (n < 32) {
        keys[n] = key;
        vals[n++] = bytes;
    }
    return cudaSuccess;
}

}  // namespace pm
