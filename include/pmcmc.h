/*
 * pmcmc.h -- C ABI of a single-GPU (GB300, sm_103a) parallel-Newton MCMC solver.
 *
 * The library evaluates an MCMC chain s_1..s_T in parallel across its length, following
 * "Parallelizing MCMC Across the Sequence Length" (arXiv 2508.18413).  With the per-step noise
 * (xi_t, u_t) fixed, the chain is the fixed point of s_t = f_t(s_{t-1}) (Section 2, Section 3).
 * Each Newton iteration (Algorithm 1)
 *   (a) evaluates f_t and a Jacobian J_t at the previous iterate for all t at once
 *       (Eq. 2: dense J = DEER; Eq. 4: diagonal = quasi-DEER; Appendix A.3: block quasi-DEER),
 *   (b) solves the linearised recursion delta_t = J_t delta_{t-1} + r_t,
 *       r_t = f_t(s_{t-1}) - s_t, with a single-pass parallel scan over affine maps (Section 2),
 *       and sets s <- s + delta (algebraically Eq. 3),
 *   (c) stops when the residual of Eq. 1 meets the tolerance.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" must be device memory of the context's GPU; "host" pointers are
 *     ordinary host memory.  The caller owns every buffer it passes; the library owns only its
 *     internal workspace (allocated lazily, reused, freed by pmcmc_destroy).
 *   - Real-valued device buffers hold double for PMCMC_F64 and float for the FP32 precisions,
 *     except u (the accept uniforms), which is always double.  Arrays are row-major with the
 *     time index slowest: s[t][d] is s + t*D + d for t = 0..T-1 (t = 0 is step 1).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is stream-ordered;
 *     calls that fill a host result struct synchronise that stream before returning.
 *   - Errors are returned as pmcmc_status; nothing is thrown across the ABI.  After a negative
 *     status, pmcmc_last_error() describes the failure.  A context is not thread-safe: use one
 *     context per host thread.
 */
#ifndef PMCMC_H
#define PMCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmcmc_ctx pmcmc_ctx;

typedef enum {
    PMCMC_OK = 0,
    PMCMC_NOT_CONVERGED = 1, /* max_iters reached; the last iterate is still written (early
                                stopping, Section 3.4) */
    PMCMC_EINVAL = -1,       /* invalid argument (sizes, NULL pointers, unsupported combination) */
    PMCMC_ENOMEM = -2,       /* workspace allocation failed */
    PMCMC_ECUDA = -3,        /* a CUDA call failed */
    PMCMC_ETIMEOUT = -4,     /* a bounded device-side wait ran out (scan look-back) */
    PMCMC_ENAN = -5,         /* the initial state or data is not finite */
    PMCMC_EUNSUPPORTED = -6  /* a size beyond what the kernels are compiled for */
} pmcmc_status;

/* f_t: the sampler transition (Section 3.2 MALA; Algorithm 2 HMC with a sequential leapfrog;
 * HMC with the leapfrog itself solved by block quasi-DEER, Section 3.3). */
typedef enum {
    PMCMC_MALA = 0,
    PMCMC_HMC = 1,
    PMCMC_HMC_PAR_LEAPFROG = 2,
    PMCMC_GIBBS = 3  /* reparameterised Gibbs sweep (Section 3.1) of the PMCMC_SCHOOLS model */
} pmcmc_sampler;

/* Built-in target densities (log p up to a constant):
 *   GAUSSIAN: -1/2 (x - mean)^T prec (x - mean)
 *   LOGREG:   sum_n [y_n z_n - log(1 + exp z_n)] - |x|^2 / (2 prior_scale^2),  z = X x
 *   BANANA:   -x1^2/200 - (x2 + 0.1 x1^2 - 10)^2 / 2   (D = 2)
 *   SCHOOLS:  the hierarchical Gaussian model of the Gibbs experiment (Appendix B.2): S schools
 *             of N scores (X: S x N, row s = school s), state (tau^2, mu, theta_1..S,
 *             sigma^2_1..S), D = 2 + 2S, 1 <= S <= 15, hyperparameters nu0 = 0.1,
 *             tau0^2 = 100, mu0 = 0, kappa0 = 0.1, alpha0 = 0.1, sigma0^2 = 10.  Sampled by
 *             PMCMC_GIBBS only.  The sweep's noise xi_t (D values, in the state's order) is the
 *             reparameterisation input: xi[0] an Inv-chi^2(nu0 + S + 1, 1) variate, xi[1] and
 *             xi[2 + s] standard normals, xi[2 + S + s] Inv-chi^2(alpha0 + N, 1) variates (the
 *             caller draws them; the seed-driven generator makes only normals and uniforms).
 *             u is not used.  step is not used. */
typedef enum { PMCMC_GAUSSIAN = 0, PMCMC_LOGREG = 1, PMCMC_BANANA = 2, PMCMC_SCHOOLS = 3 } pmcmc_target_kind;

/* Newton Jacobian used in step (a):
 *   DENSE      the full stop-gradient Jacobian (DEER, Eq. 2);
 *   DIAG       its exact diagonal (quasi-DEER, Eq. 4);
 *   BLOCK2     diagonal of each block of the leapfrog Jacobian (Appendix A.3; only
 *              PMCMC_HMC_PAR_LEAPFROG);
 *   DIAG_HUTCH one-sample Hutchinson estimate z (.) (J z), z Rademacher (Eq. 9), a new probe
 *              per Newton iteration k: z_d of step t (0-based) is bit d mod 32 of output word
 *              (d mod 128) div 32 of Philox4x32-10 at counter (d div 128, t, chain_id, 2 + k),
 *              key (low, high 32 bits of seed); a set bit gives +1, a clear bit -1;
 *   ZERO       J = 0: the plain fixed-point (Picard-type) iteration. */
typedef enum {
    PMCMC_JAC_DENSE = 0,
    PMCMC_JAC_DIAG = 1,
    PMCMC_JAC_BLOCK2 = 2,
    PMCMC_JAC_DIAG_HUTCH = 3,
    PMCMC_JAC_ZERO = 4
} pmcmc_jac;

/* Arithmetic: F64 everywhere; F32 states/f/J with the MH log-ratio's log-likelihood difference
 * accumulated in compensated FP32 and the ratio and its comparison with log u in FP64;
 * F32_SCAN_BF16 as F32 but the scan's affine pairs stored as bfloat16 and combined in FP32, and
 * for DENSE Jacobians (4 < D <= 32) the D x D compositions of the scan run on the tensor cores
 * with bfloat16 operands and FP32 accumulation (the Newton loop refines the solve; r_t is
 * always formed in FP32). */
typedef enum { PMCMC_F64 = 0, PMCMC_F32 = 1, PMCMC_F32_SCAN_BF16 = 2 } pmcmc_precision;

typedef struct {
    pmcmc_target_kind kind;
    int D;               /* dimension of x */
    int N;               /* LOGREG: number of rows of X; SCHOOLS: scores per school */
    const void *mean;    /* GAUSSIAN: D reals, device */
    const void *prec;    /* GAUSSIAN: D x D precision matrix (symmetric), row-major, device */
    const void *X;       /* LOGREG: N x D design, row-major, device; SCHOOLS: S x N scores */
    const void *y;       /* LOGREG: N labels in {0, 1}, reals, device */
    double prior_scale;  /* LOGREG: prior N(0, prior_scale^2 I) */
    const void *Q;       /* optional D x D orthogonal basis, row-major, device; the Newton solve
                            runs in z = Q^T s (Section 3.4, Eq. 10), so a diagonal Jacobian is
                            taken of Q^T J Q.  The chain is unchanged: the noise is rotated with
                            it (xi' = Q^T xi), which leaves MALA and HMC exactly equivariant.
                            Used by pmcmc_solve and pmcmc_solve_batched for GAUSSIAN and LOGREG
                            targets; NULL = identity. */
} pmcmc_target;

typedef struct {
    pmcmc_sampler sampler;
    double step;          /* step size epsilon */
    int leapfrog_L;       /* leapfrog steps per HMC transition */
    pmcmc_jac jac;
    pmcmc_precision precision;
    double atol, rtol;    /* converged when max_{t,d} (|r_td| - rtol |s_td|) <= atol (App. B) */
    int max_iters;        /* Newton updates allowed; <= 0 means T (the proven bound) */
    double damping;       /* J <- damping J before clipping; 0 means 1 (App. B.4) */
    int clip;             /* 1: clip entries of J to [-1, 1] (App. B.4) */
    int gate_grad;        /* 1: J carries the stop-gradient gate term of Section 3.2 */
    unsigned long long seed; /* noise seed when xi/u are NULL, and for Hutchinson probes */
    unsigned int chain_id;   /* noise counter of this chain */
    int spin_limit;       /* look-back wait bound (polls); 0 = default */
    int engine;           /* 0: automatic (tensor cores where a kernel exists: MALA on LOGREG,
                             F32, D <= 32, DIAG or DENSE with gate_grad 0, or ZERO, for the
                             evaluate pass; the DENSE Jacobian of MALA on LOGREG, F32, D <= 32;
                             the adjoint's dense Jacobians on LOGREG, F32, 64 < D <= 128);
                             1: CUDA cores only.  The dense scan of F32_SCAN_BF16 composes on
                             the tensor cores either way. */
    int seq_after;        /* pmcmc_solve_batched: 0 = off; > 0 = a chain not converged after
                             this many Newton sweeps is completed by the sequential loop */
    int window;           /* pmcmc_solve: 0 = off; W > 0 = sliding-window updates (Section 3.4):
                             each Newton iteration evaluates and updates only the W steps from
                             the first step not yet converged, so the Jacobian and residual
                             buffers hold W (not T) steps.  Not with Q or HMC_PAR_LEAPFROG. */
} pmcmc_options;

typedef struct {
    int iters;            /* Newton updates applied */
    int status;           /* pmcmc_status of the solve */
    double max_residual;  /* max_{t,d} |r_td| of the returned iterate */
    double accept_rate;   /* fraction of accepted MH steps in the returned iterate */
    double min_margin;    /* min_t |log alpha_t - log u_t| of the returned iterate */
    int nonfinite_resets; /* elements of an iterate that were non-finite and were reset */
    float elapsed_ms;     /* device time of the solve (CUDA events) */
    int sequential;       /* pmcmc_solve_batched with seq_after: 1 if the chain was completed by
                             the sequential loop (its s_out is then the exact sequential chain) */
} pmcmc_result;

/* Fill `opt` with defaults: MALA, step 0.01, DIAG, F32, atol 1e-5, rtol 0, max_iters T,
 * damping 1, no clip, gate_grad 1, seed 0, chain 0, engine 0. */
void pmcmc_options_default(pmcmc_options *opt);

/* Create a context on CUDA device `device`.  Returns EINVAL/ECUDA on failure. */
pmcmc_status pmcmc_create(pmcmc_ctx **ctx, int device);

/* Free the context and its workspace.  NULL is accepted. */
pmcmc_status pmcmc_destroy(pmcmc_ctx *ctx);

/* Text of the last error on this context (static storage owned by the context). */
const char *pmcmc_last_error(pmcmc_ctx *ctx);

/*
 * Counter-based noise (Section 3.2: xi_t ~ N(0, I), u_t ~ U(0, 1) are inputs of f_t).
 * Philox4x32-10 keyed by the 64-bit seed; xi[t][2j], xi[t][2j+1] are the Box-Muller pair of
 * the two 53-bit uniforms of counter (j, t, chain_id, 0); u[t] is the first 53-bit uniform of
 * counter (0, t, chain_id, 1); uniforms are (k + 1/2) 2^-53.
 *   xi: T x D device reals of `precision` (may be NULL); u: T device doubles (may be NULL).
 */
pmcmc_status pmcmc_gen_noise(pmcmc_ctx *ctx, unsigned long long seed, unsigned int chain_id,
                             int T, int D, pmcmc_precision precision, void *xi, double *u,
                             void *stream);

/*
 * Parallel Newton solve of the chain (Algorithm 1 with the update of Eq. 2/3/4).
 *   s0:     D device reals, the given initial state (Section 2).
 *   s_init: T x D device reals, the initial guess s^(0); NULL means s^(0)_t = s0 for all t
 *           (Appendix B).  Passing any iterate resumes from it.
 *   xi, u:  T x D device reals and T device doubles of noise; both NULL means generated from
 *           (opt->seed, opt->chain_id) as pmcmc_gen_noise does.
 *   s_out:  T x D device reals, written with the returned iterate (also when NOT_CONVERGED).
 *   res:    host struct filled on return (may be NULL).
 * For PMCMC_HMC_PAR_LEAPFROG the chain is solved step by step and each step's L leapfrog
 * updates are solved by block quasi-DEER (Algorithm 2); opt->max_iters then bounds the inner
 * Newton iterations per step (<= 0 means L).
 * Returns OK, NOT_CONVERGED or an error.
 */
pmcmc_status pmcmc_solve(pmcmc_ctx *ctx, const pmcmc_target *target, const pmcmc_options *opt,
                         int T, const void *s0, const void *s_init, const void *xi,
                         const double *u, void *s_out, pmcmc_result *res, void *stream);

/*
 * The sequential chain s_t = f_t(s_{t-1}) on the GPU (the paper's sequential baseline,
 * Section 5: one dependent step after another).  Same arguments as pmcmc_solve without the
 * Newton controls.  accept_out (T bytes, device, may be NULL) receives the decisions.
 */
/*
 * pmcmc_solve without a host synchronisation: the whole Newton loop is enqueued on `stream` (the
 * device-side loop of a conditional CUDA graph) followed by a kernel that writes the result to
 * res_dev, a pmcmc_result in DEVICE memory; the call returns once the work is enqueued.  The
 * solve's outcome (PMCMC_OK, PMCMC_NOT_CONVERGED, PMCMC_ENAN, PMCMC_ETIMEOUT) is in
 * res_dev->status; the return value reports argument and launch errors only (PMCMC_EUNSUPPORTED
 * with Q, PMCMC_HMC_PAR_LEAPFROG, a window, profiling on, or where conditional graphs are not
 * available).  res_dev->elapsed_ms is 0.  s_out, xi, u and res_dev must stay valid, and the
 * context unused by other calls, until the stream has passed this call.
 */
pmcmc_status pmcmc_solve_async(pmcmc_ctx *ctx, const pmcmc_target *target, const pmcmc_options *opt,
                               int T, const void *s0, const void *s_init, const void *xi,
                               const double *u, void *s_out, pmcmc_result *res_dev, void *stream);

pmcmc_status pmcmc_seq_solve(pmcmc_ctx *ctx, const pmcmc_target *target,
                             const pmcmc_options *opt, int T, const void *s0, const void *xi,
                             const double *u, void *s_out, unsigned char *accept_out,
                             void *stream);

/*
 * One evaluate-and-linearise pass (step (a)) at a given trajectory s (T x D device reals):
 *   f_out   T x D device reals: f_t(s_{t-1}) (s_{-1} = s0);
 *   jac_out device reals: T x D for DIAG/DIAG_HUTCH/ZERO, T x D x D (row-major) for DENSE;
 *           damping and clip applied (may be NULL);
 *   acc_out T device bytes: the accept decision of each step (may be NULL);
 *   ell_out T device doubles: MALA log-ratio / HMC H0 - HL before min(0, .) (may be NULL).
 * DIAG_HUTCH uses the probes of Newton iteration 0 (see pmcmc_jac).
 */
pmcmc_status pmcmc_linearize(pmcmc_ctx *ctx, const pmcmc_target *target,
                             const pmcmc_options *opt, int T, const void *s0, const void *s,
                             const void *xi, const double *u, void *f_out, void *jac_out,
                             unsigned char *acc_out, double *ell_out, void *stream);

/*
 * The parallel affine scan alone (step (b), Section 2): for t = 0..T-1,
 *   delta_t = a_t (.) delta_{t-1} + b_t  (delta_{-1} = 0),   s_t <- s_t + delta_t.
 * kind PMCMC_JAC_DIAG: a, b are T x D (elementwise maps, quasi-DEER Eq. 4);
 * kind PMCMC_JAC_DENSE: a is T x D x D row-major (a_t delta is a matrix-vector product), b T x D,
 *   D <= 32 (F32_SCAN_BF16: 4 < D <= 32, the compositions of a on the tensor cores).
 * precision: F64 (a, b, s double), F32 (float), F32_SCAN_BF16 (a, b bfloat16, s float).
 * s: T x D device, updated in place.  Single pass, decoupled look-back.
 * The diagonal kernel (D <= 32) is chosen from T D, D and the precision; these environment
 * variables, read at every call (comparisons, tests), override the choice: PMCMC_SCAN_KERNEL =
 * rows | staged | pipe | cluster (staged, pipe and cluster need a, b, s 16-byte aligned and
 * cluster FP32 or F32_SCAN_BF16, else the row kernel runs); PMCMC_SCAN_SHAPE = "rows,sub-chunks" (rows 8 or 16) for the row
 * kernel; PMCMC_SCAN_DCONST = 0 keeps the row kernel's generic instance for every D;
 * PMCMC_PIPE_CTAS = 2 runs two pipelined CTAs per SM; PMCMC_SCAN_CLUSTER = 2 | 4 | 8,
 * PMCMC_SCAN_SLOTS = 4 | 8 and PMCMC_SCAN_LAG shape the cluster kernel.  Results differ only by
 * the association of the FP arithmetic.
 */
pmcmc_status pmcmc_scan(pmcmc_ctx *ctx, pmcmc_jac kind, pmcmc_precision precision, int T, int D,
                        const void *a, const void *b, void *s, void *stream);

/*
 * The kernel pmcmc_scan would run for a diagonal scan (kind PMCMC_JAC_DIAG) of T x D at
 * `precision` with 16-byte-aligned a, b and s, computed on the host without device work (the
 * same environment variables are read):
 *   kernel_out     0 row kernel (D a run-time value), 1 row kernel with D fixed at compile time,
 *                  2 register-resident kernel (one sub-chunk per warp), 3 staged bulk copies,
 *                  4 pipelined bulk copies, 5 thread-block cluster, 6 shared-memory kernel (D > 32);
 *   tile_out       timesteps per tile (per cluster tile for 5);
 *   tiles_out      tiles of the launch;
 *   max_tiles_out  tiles the look-back workspace of pmcmc_scan holds (a launch needs
 *                  tiles_out <= max_tiles_out).
 * PMCMC_EINVAL for T or D <= 0, a null output or an unknown precision; PMCMC_EUNSUPPORTED for
 * another kind or D > 256.  Needs no context and no GPU.
 */
pmcmc_status pmcmc_scan_plan(pmcmc_jac kind, pmcmc_precision precision, int T, int D, int *kernel_out,
                             int *tile_out, int *tiles_out, int *max_tiles_out);

/*
 * Adjoint of a chain functional at the converged fixed point, with every accept decision held
 * (the chain is then a smooth function of the parameters).  Given dL/ds (T x D device reals)
 * it runs the transposed recursion backward,
 *   lambda_t = dL/ds_t + J_{t+1}^T lambda_{t+1},   lambda_T = dL/ds_T,
 * as a parallel reverse scan with dense J_{t+1} = I + step H(s_t) (accepted) or I (rejected),
 * and returns dL/dtheta = sum_t lambda_t^T d f_t/d theta for theta = (step, prior_scale).
 * J is recomputed in segments when T*D*D reals exceed jac_budget_bytes (0 = no limit).
 * PMCMC_MALA with LOGREG (D <= 128 in FP32, 64 in FP64) or GAUSSIAN targets.  With LOGREG in
 * FP32 and 64 < D <= 128 the J's are formed on the tensor cores (split-tf32 products of FP32
 * accuracy; opt->engine = 1 selects the CUDA-core kernel).  The workspace then also holds an
 * image of X^T of 32 KiB per 32 data rows.
 * s: the converged trajectory; acc: its T decisions (device bytes); u is not used (the
 * decisions are given).  lambda_out (T x D device reals, may be NULL) receives lambda.
 * grad_out: 2 host doubles, dL/dstep and dL/dprior_scale (zero for Gaussian targets).
 */
pmcmc_status pmcmc_adjoint(pmcmc_ctx *ctx, const pmcmc_target *target, const pmcmc_options *opt,
                           int T, const void *s0, const void *s, const unsigned char *acc,
                           const void *xi, const double *u, const void *dL_ds,
                           size_t jac_budget_bytes, void *lambda_out, double *grad_out,
                           void *stream);

/*
 * The diagonal scan of pmcmc_scan (kind PMCMC_JAC_DIAG) without any allocation and without a
 * context.  The paper has no counterpart: this exists for callers that cannot allocate device
 * memory, such as code running during CUDA stream capture (cudaMalloc is not a stream
 * operation), hosts that fix their memory budget at start-up, and plugins inside a framework
 * whose allocator owns the device.  Its scratch (look-back flags, tile aggregates, control
 * words) is one static device array of 8 MiB that every GPU loading the library holds until
 * process exit.  The first call on a device (with it current) looks up the array's address;
 * make that call before any stream capture.  The address is kept per device ordinal for the
 * rest of the process: it belongs to the device's primary context, so call this from the
 * primary context and do not reset the device in between.  Each call clears what must start at zero with
 * cudaMemsetAsync on `stream`; it neither allocates nor frees.  All calls share the array:
 * calls that overlap on the GPU race, so order them on one stream.  The call is asynchronous
 * and does not report device-side look-back timeouts: if a bounded look-back wait runs out
 * (it does not with the default bound unless the GPU is shared with work that starves the
 * scan), the call still returns and stays within its buffers, but s is undefined.
 * Returns EINVAL for bad arguments and EUNSUPPORTED when D > 256 or the scan's scratch
 * (about 4 + 3 D r bytes per tile, r = 4 or 8, tiles of about 3300 to 4200 elements for
 * D <= 32, 4096 / D timesteps above) exceeds 8 MiB.
 */
pmcmc_status pmcmc_scan_noalloc(pmcmc_precision precision, int T, int D, const void *a,
                                const void *b, void *s, void *stream);

/* One chain of a batched solve. */
typedef struct {
    pmcmc_target target;
    pmcmc_sampler sampler; /* PMCMC_MALA or PMCMC_HMC */
    double step;
    int leapfrog_L;
    int T;
    const void *s0;        /* D device reals */
    const void *xi;        /* T x D device reals */
    const double *u;       /* T device doubles */
    void *s_out;           /* T x D device reals */
} pmcmc_chain_desc;

/*
 * Many independent chains of uneven T, D, sampler and target solved together (the batching
 * of Section 5.2) by one persistent kernel per Newton sweep, captured in a CUDA graph whose
 * device-side loop runs until every chain has converged.  Uses opt->jac (DIAG or
 * DIAG_HUTCH), opt->precision (F32 or F32_SCAN_BF16), atol/rtol, max_iters, damping, clip.
 * Per-chain results go to res (B host structs, may be NULL).
 * With opt->seq_after > 0 the Newton sweeps stop after seq_after sweeps (or max_iters, if
 * smaller), and every chain not converged by then is recomputed by the sequential loop, several
 * chains at once on separate streams; res[i].sequential marks those chains.  A chain whose
 * Newton frontier advances a few steps per sweep costs less sequentially (Section 5.2 finds the
 * same trade-off for batches).
 */
pmcmc_status pmcmc_solve_batched(pmcmc_ctx *ctx, int B, const pmcmc_chain_desc *chains,
                                 const pmcmc_options *opt, pmcmc_result *res, void *stream);

/*
 * The sequential chains of a batch on the GPU in one launch: the baseline of
 * pmcmc_solve_batched (the paper's sequential loop, Section 5, for many chains at once).  One
 * CTA per chain, the longest chains dispatched first; each chain runs its T dependent steps with
 * its design (logistic) or precision matrix (Gaussian) in shared memory.  MALA or HMC chains on
 * GAUSSIAN or LOGREG targets with D <= 128 whose design fits one SM's shared memory
 * (EUNSUPPORTED otherwise); opt->precision F32 or F64 gives the arithmetic (u is double, the
 * accept decision is taken in FP64).  Target Q, Newton and tolerance fields are not used.
 * chains[i].s_out (T x D device reals) receives chain i.  Asynchronous on `stream`.
 */
pmcmc_status pmcmc_seq_solve_batched(pmcmc_ctx *ctx, int B, const pmcmc_chain_desc *chains,
                                     const pmcmc_options *opt, void *stream);

/*
 * Measurement support (the paper reports post-compilation wall-clock only, Section 5 and
 * Appendix B; these counters explain such a number).  While enabled, the context counts every
 * kernel it launches and brackets each evaluate-and-linearise, dense-Jacobian and scan launch
 * with CUDA events on the launching stream, accumulating their device durations.
 * pmcmc_profile_enable(ctx, 1) resets the counters; (ctx, 0) stops recording.
 */
typedef struct {
    long long launches;       /* kernels launched by this context while enabled */
    long long eval_launches;  /* evaluate-and-linearise launches */
    double eval_ms;           /* their summed device time */
    long long jac_launches;   /* dense Jacobian assembly launches */
    double jac_ms;
    long long scan_launches;  /* scan launches */
    double scan_ms;
} pmcmc_profile;

pmcmc_status pmcmc_profile_enable(pmcmc_ctx *ctx, int enable);
pmcmc_status pmcmc_profile_get(pmcmc_ctx *ctx, pmcmc_profile *out);

#ifdef __cplusplus
}
#endif

#endif /* PMCMC_H */
