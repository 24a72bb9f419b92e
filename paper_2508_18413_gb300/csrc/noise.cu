// Counter-based sampler noise (xi_t ~ N(0, I), u_t ~ U(0, 1) are the inputs of f_t,
// Section 3.2).  Philox4x32-10 keyed by the 64-bit seed:
//   xi[t][2j], xi[t][2j+1]  Box-Muller pair from the two 53-bit uniforms of counter (j, t, c, 0)
//   u[t]                    first 53-bit uniform of counter (0, t, c, 1)
// One thread per (t, j) pair; FP64 Box-Muller, rounded once to the output type.
#include "common.cuh"
#include "internal.h"

namespace pm {

template <typename R>
__global__ void __launch_bounds__(256) noise_kernel(unsigned long long seed, unsigned int chain,
                                                    int T, int D, R *__restrict__ xi,
                                                    double *__restrict__ u) {
    const int P = (D + 1) >> 1;
    const long long total = (long long)T * (P + 1);
    const uint2 key = make_uint2((unsigned int)seed, (unsigned int)(seed >> 32));
    const double two_pi = 6.283185307179586476925286766559;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(i / (P + 1));
        const int j = (int)(i - (long long)t * (P + 1));
        if (j < P) {
            if (!xi) continue;
            uint4 w = philox4x32_10(make_uint4((unsigned int)j, (unsigned int)t, chain, 0u), key);
            double u1 = uniform53(w.x, w.y), u2 = uniform53(w.z, w.w);
            double r = sqrt(-2.0 * log(u1));
            double s, c;
            sincos(two_pi * u2, &s, &c);
            R *row = xi + (size_t)t * D;
            row[2 * j] = (R)(r * c);
            if (2 * j + 1 < D) row[2 * j + 1] = (R)(r * s);
        } else {
            if (!u) continue;
            uint4 w = philox4x32_10(make_uint4(0u, (unsigned int)t, chain, 1u), key);
            u[t] = uniform53(w.x, w.y);
        }
    }
}

cudaError_t launch_noise(unsigned long long seed, unsigned int chain, int T, int D, bool f64,
                         void *xi, double *u, cudaStream_t st) {
    const long long total = (long long)T * ((D + 1) / 2 + 1);
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (blocks < 1) blocks = 1;
    if (f64)
        noise_kernel<double><<<blocks, 256, 0, st>>>(seed, chain, T, D, (double *)xi, u);
    else
        noise_kernel<float><<<blocks, 256, 0, st>>>(seed, chain, T, D, (float *)xi, u);
    return cudaGetLastError();
}

}  // namespace pm
