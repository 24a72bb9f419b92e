// Arguments of the evaluate-and-linearise kernels (step (a) of a Newton iteration).
#pragma once

#include <cuda_runtime.h>

#include "../../include/pmcmc.h"

namespace pm {

struct EvalStats;
struct ScanCtl;
struct CtlBlock;

struct EvalArgs {
    // problem
    int target = 0;      // pmcmc_target_kind
    int sampler = 0;     // pmcmc_sampler
    int T = 0, D = 0, L = 0, N = 0;
    double eps = 0.0;
    double sigma_p = 1.0;
    int jac = PMCMC_JAC_DIAG;
    int gate_grad = 1;
    double damping = 1.0;
    int clip = 0;
    double rtol = 0.0;
    bool f64 = false;    // arithmetic type double (else float)
    bool bf16 = false;   // scan pair storage bfloat16 (FP32 arithmetic)
    // inputs (device)
    const void *s0 = nullptr;   // D
    const void *s = nullptr;    // T x D current iterate
    const void *xi = nullptr;   // T x D
    const double *u = nullptr;  // T
    const void *mu = nullptr;   // Gaussian mean
    const void *P = nullptr;    // Gaussian precision
    const void *X = nullptr;    // logistic design N x D
    const void *Xp = nullptr;   // logistic design, padded copy (workspace)
    const void *y = nullptr;    // logistic labels
    // outputs (device, optional)
    void *a_out = nullptr;      // J: T x D (diag) or T x D x D (dense)
    void *b_out = nullptr;      // r = f - s: T x D
    void *f_out = nullptr;      // f: T x D
    unsigned char *acc_out = nullptr;
    double *ell_out = nullptr;
    void *w_out = nullptr;      // logistic dense J: sigmoid'(z) per (t, n), T x N
    void *rank1_u = nullptr;    // logistic dense J: gate term vectors, T x D each
    void *rank1_v = nullptr;
    EvalStats *stats = nullptr;
    // probes / control
    unsigned long long seed = 0;
    unsigned int chain = 0;
    const int *iter = nullptr;  // device Newton iteration counter (Hutchinson probes)
    const int *skip = nullptr;  // device flag: skip the launch when set (device-side loop)
    // tensor-core path (logistic MALA, D <= 32)
    int engine = 0;                   // pmcmc_options.engine: 0 automatic, 1 CUDA cores only
    const void *tc_img = nullptr;     // chunk images of the design (launch_logreg_tc_pack)
    unsigned int *timeout = nullptr;  // set to 1 when a bounded wait ran out
    unsigned int spin_limit = 0;      // polls per wait; 0 = default
    // tensor-core dense Jacobian (logistic MALA, D <= 32): pair image of the design
    // (launch_logreg_pair_pack); null selects the CUDA-core assembly
    const void *pair_img = nullptr;
    // Newton update fused into the tensor-core evaluate kernel (fs_flags non-null): the kernel
    // also solves delta_t = J_t delta_{t-1} + r_t (carry from the published aggregates of the
    // earlier tiles) and writes s + delta to the other iterate buffer.  The parity of *iter
    // picks the buffers: even reads s and writes s_alt, odd the reverse.
    void *s_alt = nullptr;
    unsigned int *fs_flags = nullptr;  // one per 128-timestep tile, epoch-tagged
    float *fs_agg = nullptr;           // tiles x 2 x 32: tile aggregates (A, B)
    ScanCtl *fs_ctl = nullptr;         // ticket, done, epoch, timeout
    // device-side Newton loop (fused path, inside the loop's graph): the last tile to finish
    // also takes the loop's convergence decision and sets the WHILE condition (null: a separate
    // control kernel does)
    CtlBlock *loop = nullptr;
    unsigned long long loop_handle = 0;  // cudaGraphConditionalHandle
    double loop_atol = 0.0;
    int loop_max_iters = 0;
};

cudaError_t launch_eval_small(const EvalArgs &A, cudaStream_t st);
// reparameterised Gibbs on the schools target (eval_gibbs.cu): R arithmetic, S pair storage
bool gibbs_supported(int D, int N);
template <typename R, typename S>
cudaError_t launch_gibbs(const EvalArgs &A, cudaStream_t st, bool seq);
cudaError_t launch_seq_small(const EvalArgs &A, cudaStream_t st);
cudaError_t launch_eval_logreg(const EvalArgs &A, cudaStream_t st);
cudaError_t launch_seq_logreg(const EvalArgs &A, cudaStream_t st);
cudaError_t launch_logreg_dense_jac(const EvalArgs &A, cudaStream_t st);
int logreg_padded_dim(int D);

// tensor-core evaluate-and-linearise of logistic MALA (eval_logreg_tc.cu)
bool logreg_tc_supported(const EvalArgs &A);
size_t logreg_tc_image_bytes(int N);
cudaError_t launch_logreg_tc_pack(const void *X, const void *y, int N, int D, void *img, cudaStream_t st);
cudaError_t launch_eval_logreg_tc(const EvalArgs &A, cudaStream_t st);
constexpr int kTcTileT = 128;  // timesteps per CTA of the tensor-core evaluate kernel

// tensor-core assembly of the dense logistic-MALA Jacobian (jac_logreg_tc.cu)
bool logreg_jac_tc_supported(const EvalArgs &A);
size_t logreg_pair_image_bytes(int N, int D);
cudaError_t launch_logreg_pair_pack(const void *X, int N, int D, void *img, cudaStream_t st);
cudaError_t launch_jac_logreg_tc(const EvalArgs &A, cudaStream_t st);

}  // namespace pm
