// Internal launch interfaces shared by the translation units of libpmcmc.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

#include "../../include/pmcmc.h"

namespace pm {

struct ScanCtl;
struct EvalStats;

constexpr unsigned int kDefaultSpinLimit = 1u << 22;

// Workspace for one decoupled look-back scan: per-tile flags and aggregates.
struct ScanWork {
    unsigned int *flags = nullptr;  // ntiles, zero-initialised once
    void *agg = nullptr;            // ntiles * (D*D + D) reals (dense) or 2*D (diag)
    void *incl = nullptr;           // ntiles * D reals
    int max_tiles = 0;
    ScanCtl *ctl = nullptr;
};

// Tile geometry of the diagonal scan for (T, D): timesteps per tile.
int diag_scan_tile(int T, int D, int elem_bytes);
int dense_scan_chunk(int T, int D);
int diag_scan_tile_rows(int T, int D);
void scan_shape_override(int rows, int nsub);

cudaError_t launch_noise(unsigned long long seed, unsigned int chain, int T, int D, bool f64,
                         void *xi, double *u, cudaStream_t st);

// storage: 0 = same as arithmetic, 1 = bfloat16 (FP32 arithmetic only)
cudaError_t launch_scan_diag(bool f64, int storage, int T, int D, int tile_t, const void *a,
                             const void *b, void *s, const void *s_reset, const ScanWork &w,
                             EvalStats *stats, const int *skip, unsigned int spin_limit,
                             cudaStream_t st);

// The diagonal-scan kernel launch_scan_diag picks (a, b, s 16-byte aligned), without device work.
enum ScanPlanKernel {
    kPlanRows = 0,         // row kernel, D a run-time value
    kPlanRowsConstD = 1,   // row kernel, D fixed at compile time
    kPlanRegister = 2,     // register-resident kernel, one sub-chunk per warp
    kPlanStaged = 3,       // bulk copies into shared memory
    kPlanPipe = 4,         // persistent, double-buffered bulk copies
    kPlanCluster = 5,      // tiles shared by a thread-block cluster
    kPlanDiagWide = 6      // shared-memory staged kernel for D > 32
};
void plan_scan_diag(bool f64, int storage, int T, int D, int *kernel, int *tile, int *tiles);

// Row kernel of the diagonal scan with D a compile-time constant (D a power of two up to 32,
// 8 rows per warp, `nsub` sub-chunks per warp); kind 0: FP32, 1: FP32 with bfloat16 a and b,
// 2: FP64.  cudaErrorInvalidValue for any other D or a tile count beyond the workspace.
cudaError_t launch_scan_rows_dconst(int kind, int T, int D, int nsub, const void *a, const void *b, void *s,
                                    const void *s_reset, const ScanWork &w, EvalStats *stats,
                                    const int *skip, unsigned int spin_limit, cudaStream_t st);

// Diagonal scan on thread-block clusters (FP32 iterates, D <= 32, a, b and s 16-byte aligned;
// storage 1: a and b bfloat16).
int diag_scan_tile_cluster(int D, int sbytes);
cudaError_t launch_scan_diag_cluster(int storage, int T, int D, const void *a, const void *b, void *s,
                                     const void *s_reset, const ScanWork &w, EvalStats *stats,
                                     const int *skip, unsigned int spin_limit, cudaStream_t st);

// Dense scan with the compositions on the tensor cores (bfloat16 products, FP32 accumulation),
// 4 < D <= 32: b bfloat16; a bfloat16 (a_bf16) or float.  Tiles of 4 chunks of `chunk` steps.
int dense_tc_chunk(int T);
cudaError_t launch_scan_dense_tc(bool a_bf16, int T, int D, int chunk, const void *a, const void *b,
                                 void *s, const void *s_reset, const ScanWork &w, EvalStats *stats,
                                 const int *skip, unsigned int spin_limit, cudaStream_t st);

cudaError_t launch_scan_dense(bool f64, int T, int D, int chunk, const void *a, const void *b,
                              void *s, const void *s_reset, const ScanWork &w, EvalStats *stats,
                              const int *skip, unsigned int spin_limit, cudaStream_t st);

}  // namespace pm
