// FP32 arithmetic with bfloat16 storage of the scan pairs (J_t, r_t).
#include "eval_small.cuh"

namespace pm {

cudaError_t launch_eval_small_bf16(const EvalArgs &A, cudaStream_t st) {
    return dispatch_ts<float, __nv_bfloat16>(A, st, false);
}

}  // namespace pm
