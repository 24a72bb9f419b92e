// FP64 instantiations of the per-thread evaluate-and-linearise pass.
#include "eval_small.cuh"

namespace pm {

cudaError_t launch_eval_small_f64(const EvalArgs &A, cudaStream_t st) {
    return dispatch_ts<double, double>(A, st, false);
}

cudaError_t launch_seq_small_f64(const EvalArgs &A, cudaStream_t st) {
    return dispatch_ts<double, double>(A, st, true);
}

}  // namespace pm
