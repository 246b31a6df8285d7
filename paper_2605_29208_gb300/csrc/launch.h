// Launchers of the templated inference kernels (one translation unit per
// kernel family so that the builds compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "estep_small.cuh"
#include "viterbi_small.cuh"

namespace hmm {

// Chain shapes compiled for the small-N kernels: (padded N, lanes per chain).
bool estep_small_supported(int NP, int G);
bool viterbi_small_supported(int NP, int G);
int default_estep_G(int NP, int64_t n_seq, int n_sm);
int default_viterbi_G(int NP, int64_t n_seq, int n_sm);

// Sequences per work item of each kernel.
inline int estep_seqs_per_item(int G) { return 16 / G; }
inline int viterbi_seqs_per_item(int G) { return 32 / G; }

constexpr int kWarpsPerBlock = 4;

// mode: MODE_STATS | MODE_GAMMA (0 is treated as MODE_STATS); fam: the batch's
// single family, FAM_TABLE (log b table) or FAM_ANY (mixed families)
cudaError_t launch_estep_small(int NP, int G, int mode, const EStepArgs& a, int fam, int n_sm,
                               cudaStream_t st);
// per-NP translation units
cudaError_t launch_estep_np2_4(int NP, int G, int mode, const EStepArgs& a, int fam, int n_sm,
                               cudaStream_t st);
cudaError_t launch_estep_np8(int G, int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st);
cudaError_t launch_estep_np16(int G, int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st);
cudaError_t launch_estep_np32(int G, int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st);
cudaError_t launch_viterbi_small(int NP, int G, const VitArgs& a, int fam, int n_sm,
                                 cudaStream_t st);

}  // namespace hmm
