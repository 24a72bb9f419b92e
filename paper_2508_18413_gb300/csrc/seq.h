// The sequential chain on the GPU (seq.cu): one CTA, or one cluster of CTAs, per chain.
#pragma once

#include <cuda_runtime.h>

#include "../../include/pmcmc.h"
#include "eval.h"

namespace pm {

constexpr int kSeqDMax = 128;             // largest state dimension
constexpr int kSeqThreads = 512;          // threads per CTA of a single-chain launch
constexpr int kSeqThreadsBatched = 256;   // threads per CTA of a many-chain launch
constexpr size_t kSeqSmemBudget = 220 * 1024;  // dynamic shared memory per CTA

// One chain (MALA or HMC on a Gaussian or logistic-regression target).  Pointers are device
// memory of the arithmetic type (double or float; u always double).
struct SeqChain {
    int target = 0, sampler = 0, D = 0, N = 0, L = 0, T = 0;
    double eps = 0.0, sigma_p = 1.0;
    const void *X = nullptr, *y = nullptr, *mu = nullptr, *P = nullptr;
    const void *s0 = nullptr, *xi = nullptr;
    const double *u = nullptr;
    void *s_out = nullptr;
    unsigned char *acc_out = nullptr;
};

SeqChain seq_chain_from(const EvalArgs &A);  // the chain of a sequential-loop launch
bool seq_fast_supported(const SeqChain &ch);
size_t seq_smem_bytes(const SeqChain &ch, int cs, int threads, bool f64);
int seq_cluster_size(const SeqChain &ch, bool f64);
// one chain, a cluster of seq_cluster_size() CTAs
cudaError_t launch_seq_chain(const SeqChain &ch, bool f64, cudaStream_t st);
// B chains (device array), one CTA of kSeqThreadsBatched threads each, smem bytes per CTA
cudaError_t launch_seq_chains(const SeqChain *dev_chains, int B, size_t smem, bool f64,
                              cudaStream_t st);

}  // namespace pm
