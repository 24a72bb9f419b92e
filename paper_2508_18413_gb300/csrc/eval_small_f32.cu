// FP32 instantiations of the per-thread evaluate-and-linearise pass and the dispatcher.
#include "eval_small.cuh"

namespace pm {

cudaError_t launch_eval_small_f64(const EvalArgs &A, cudaStream_t st);
cudaError_t launch_eval_small_bf16(const EvalArgs &A, cudaStream_t st);
cudaError_t launch_seq_small_f64(const EvalArgs &A, cudaStream_t st);

cudaError_t launch_eval_small(const EvalArgs &A, cudaStream_t st) {
    if (A.f64) return launch_eval_small_f64(A, st);
    if (A.bf16) return launch_eval_small_bf16(A, st);
    return dispatch_ts<float, float>(A, st, false);
}

cudaError_t launch_seq_small(const EvalArgs &A, cudaStream_t st) {
    if (A.f64) return launch_seq_small_f64(A, st);
    return dispatch_ts<float, float>(A, st, true);
}

}  // namespace pm
