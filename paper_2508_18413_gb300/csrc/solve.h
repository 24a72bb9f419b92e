// Host-side state shared by the translation units of libpmcmc.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>

#include "common.cuh"
#include "eval.h"
#include "internal.h"

namespace pm {

constexpr int kMaxStats = 4;

// Device control block of a context (one per context, never reallocated).
struct CtlBlock {
    ScanCtl scan;
    EvalStats stats[kMaxStats];
    int iter;             // Newton iteration index (read by the Hutchinson probes)
    int nonfinite_input;  // set when s0 or the initial guess is not finite
    int converged;
    int skip;             // device-side loop: set once the loop is finished
    int iters_done;
    int first_bad;        // sliding window: first step of the window not yet converged
    int win_accepts;      // sliding window: accepted steps of the frozen prefix
    int pad;
    unsigned long long inner_iters;  // parallel leapfrog: inner Newton iterations, all steps
    unsigned long long inner_max;
};

// One step of the device-side control of the Newton loop (Algorithm 1): decides convergence from
// the residual statistics of the evaluation just finished, keeps them for the host, and sets
// the WHILE condition of the graph (1: another iteration; 0: stop).  Called by a one-thread
// kernel after the evaluate pass, or by the last tile of the fused evaluate-and-update kernel.
__device__ inline void loop_control_step(CtlBlock *c, cudaGraphConditionalHandle h, double atol,
                                         int max_iters) {
    EvalStats &s = c->stats[0];
    EvalStats &keep = c->stats[1];
    keep.err = s.err;
    keep.rmax = s.rmax;
    keep.min_margin = s.min_margin;
    keep.accepts = s.accepts;
    const bool conv = ord_decode(s.err) <= atol;
    if (c->nonfinite_input || conv || c->iter >= max_iters || c->scan.timeout) {
        c->converged = conv && !c->nonfinite_input;
        c->skip = 1;
        cudaGraphSetConditional(h, 0);
    } else {
        c->iter += 1;
        c->skip = 0;
        s.err = kOrdNegInf;
        s.rmax = 0x8000000000000000ull;
        s.min_margin = 0xfff0000000000000ull;
        s.accepts = 0;
        cudaGraphSetConditional(h, 1);
    }
}

// Bump allocator over the context workspace (offsets, 256-byte aligned).
struct Carve {
    size_t used = 0;
    size_t take(size_t bytes);
};

}  // namespace pm

struct pmcmc_ctx {
    int device = 0;
    std::string err;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    unsigned long long ws_generation = 0;
    pm::CtlBlock *ctl = nullptr;       // device
    pm::CtlBlock *host_ctl = nullptr;  // pinned host mirror
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;          // device-side Newton loop (conditional WHILE node)
    cudaGraphExec_t graph_exec = nullptr;
    std::string graph_key;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t seq_streams[16] = {};  // batched: concurrent sequential completions
    cudaEvent_t seq_events[17] = {};
    int no_graph = 0;
    unsigned long long flags_generation = ~0ull;
    size_t flags_offset = 0, flags_zeroed = 0;
    unsigned long long resets_accum = 0;
    // measurement (pmcmc_profile_*)
    int prof_on = 0;
    pmcmc_profile prof{};
    cudaEvent_t pev[6] = {};
    // batched solver: autotuned shapes and the captured persistent launch
    std::map<std::string, std::pair<int, int>> tune_cache;
    void *aux = nullptr;  // rotated copies for the orthogonal basis Q
    size_t aux_bytes = 0;
    void *seq_desc = nullptr;  // chain descriptors of a many-chain sequential launch
    size_t seq_desc_bytes = 0;
    std::string batch_graph_key;
    cudaGraphExec_t batch_graph_exec = nullptr;
};

namespace pm {

pmcmc_status ws_reserve(pmcmc_ctx *c, size_t bytes);
pmcmc_status check_problem(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                           const void *s0, bool sequential);
void fill_eval_args(EvalArgs &A, const pmcmc_target *tg, const pmcmc_options *o, int T);
pmcmc_status newton_solve(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                          const void *s0, const void *s_init, const void *xi, const double *u,
                          void *s_out, pmcmc_result *res, void *stream,
                          pmcmc_result *res_dev = nullptr);
pmcmc_status window_solve(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                          const void *s0, const void *s_init, const void *xi, const double *u,
                          void *s_out, pmcmc_result *res, void *stream);
pmcmc_status solve_par_leapfrog(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o,
                                int T, const void *s0, const void *xi, const double *u,
                                void *s_out, pmcmc_result *res, void *stream);
pmcmc_status set_error(pmcmc_ctx *c, pmcmc_status st, const char *msg);
pmcmc_status solve_with_basis(pmcmc_ctx *c, const pmcmc_target *tg, const pmcmc_options *o, int T,
                              const void *s0, const void *s_init, const void *xi, const double *u,
                              void *s_out, pmcmc_result *res, void *stream);
pmcmc_status aux_reserve(pmcmc_ctx *c, size_t bytes);
cudaError_t rot_rows(void *dst, const void *src, const void *Q, long long rows, int D,
                     bool transpose, bool f64, cudaStream_t st);
cudaError_t rot_sym(void *out, const void *P, const void *Q, int D, bool f64, cudaStream_t st);
cudaError_t pad_rows_launch(void *dst, const void *src, int N, int D, int Npad, int DP, int esz,
                            cudaStream_t st);

// Profiling helpers: count a launch; bracket a timed launch (slot 0 eval, 1 jac, 2 scan).
inline void prof_count(pmcmc_ctx *c, int n = 1) {
    if (c->prof_on) c->prof.launches += n;
}
inline void prof_begin(pmcmc_ctx *c, int slot, cudaStream_t st) {
    if (c->prof_on) cudaEventRecord(c->pev[2 * slot], st);
}
inline void prof_end(pmcmc_ctx *c, int slot, cudaStream_t st) {
    if (c->prof_on) cudaEventRecord(c->pev[2 * slot + 1], st);
}
// after a stream sync: accumulate the durations of the bracketed launches
inline void prof_collect(pmcmc_ctx *c, int slot) {
    if (!c->prof_on) return;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->pev[2 * slot], c->pev[2 * slot + 1]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (slot == 0) { c->prof.eval_ms += ms; c->prof.eval_launches++; }
    if (slot == 1) { c->prof.jac_ms += ms; c->prof.jac_launches++; }
    if (slot == 2) { c->prof.scan_ms += ms; c->prof.scan_launches++; }
}

}  // namespace pm
