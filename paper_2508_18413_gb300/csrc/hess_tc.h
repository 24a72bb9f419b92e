// Tensor-core dense Jacobians of held-decision MALA steps on the logistic target (adjoint).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

namespace pm {

// 64 < D <= 128 (one 128-row MMA tile per step), FP32
bool hess_tc_supported(int D, int N);
// bytes of the X^T image (head and remainder, pre-swizzled, 32 data rows per chunk)
size_t hess_tc_image_bytes(int N);
// floats of the w workspace for nlist steps (rows padded to a multiple of 32)
size_t hess_tc_w_floats(int nlist, int N);
cudaError_t launch_hess_tc_pack(const float *X, int N, int D, void *img, cudaStream_t st);
// Jbuf[g] = I + eps H(x_g) (row-major D x D) for g < nlist, x_g = s_{list[g] - 1} (s0 for step
// 0); H = -X^T diag(w) X - inv_sp2 I.  W: workspace of hess_tc_w_floats(nlist, N) floats
// (256-byte aligned).  Sets *timeout if a bounded wait ran out.
cudaError_t launch_hess_logreg_tc(int nlist, const int *list, int D, int N, const float *X,
                                  const void *img, const float *s0, const float *s, float *W,
                                  float eps, float inv_sp2, float *Jbuf, unsigned int *timeout,
                                  unsigned int spin_limit, cudaStream_t st);

}  // namespace pm
