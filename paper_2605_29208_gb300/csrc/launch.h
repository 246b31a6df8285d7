// Launchers of the templated inference kernels (one translation unit per
// kernel family so that the builds compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "estep_small.cuh"
#include "large.cuh"
#include "viterbi_small.cuh"

namespace hmm {

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The attribute is a per-device property of the kernel and
// setting it also lowers the limit, so the largest size requested so far is
// kept per (kernel, device) and the attribute only ever grows (a kernel whose
// shared memory depends on its arguments asks for different sizes);
// thread-safe.
inline cudaError_t ensure_max_dyn_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{kernel, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Chain shapes compiled for the small-N kernels: (padded N, lanes per chain).
bool estep_small_supported(int NP, int G);
bool viterbi_small_supported(int NP, int G);
int default_estep_G(int NP, int64_t n_seq, int n_sm);
int default_viterbi_G(int NP, int64_t n_seq, int n_sm);

// Sequences per work item of each kernel.
inline int estep_seqs_per_item(int G) { return 16 / G; }
inline int viterbi_seqs_per_item(int G) { return 16 / G; }   // two chains per sequence

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
// large-N kernels (padded N in {64, 128, 256, 512, 1024})
cudaError_t launch_large_fb(int NP, const LargeArgs& a, cudaStream_t st);
cudaError_t launch_large_viterbi(int NP, const LargeArgs& a, cudaStream_t st);
// the same recursions for few groups at padded N = 256 on clusters of two
// CTAs with A resident in shared memory (the single-sequence latency path)
constexpr int LG_CL_MAX_GROUPS = 32;
bool large_cl_supported(int NP, int n_groups);
cudaError_t launch_large_fb_cl(const LargeArgs& a, cudaStream_t st);
bool large_cl1_supported(int NP, int group_fill);
cudaError_t launch_large_fb_cl1(int NP, const LargeArgs& a, cudaStream_t st);
cudaError_t launch_large_viterbi_cl1(int NP, const LargeArgs& a, cudaStream_t st);
cudaError_t launch_large_viterbi_cl(const LargeArgs& a, cudaStream_t st);
// tensor-core recursions (tcgen05, FP16 operands): padded N in {64, ..., 512},
// tiles of tc_tile_rows() sequences of one model; same outputs as launch_large_fb
bool tc_supported(int NP);
bool tc_tf32_supported(int NP);
int tc_tile_rows();
cudaError_t launch_tc_fb(int NP, const LargeArgs& a, const int32_t* tiles, int n_tiles, int* status, bool tf32,
                         cudaStream_t st);
// xi blocks on the tensor cores (TF32, K = time), padded N 128-1024: the
// transposed operands XT / YT [NP][ktot] float32 in the chunk-ordered K layout
// of the plan (kseq, kc0, kused, kpad), then the GEMM into xi_chunk
bool tc_xi_supported(int NP);
cudaError_t launch_tc_xi(const LargeArgs& a, const float* rz, const int32_t* tile_seq, const int32_t* tile_row,
                         int n_tiles, const int64_t* kseq, const int64_t* kc0, const int32_t* kused,
                         const int32_t* kpad, int n_chunks, int64_t ktot, float* XT, float* YT, double* xi_chunk,
                         int* status, cudaStream_t st);
// time-parallel forward-backward rows for small N (padded N <= 32): chunks of
// L steps, transfer matrices, boundary vectors, recomputed rows in the
// large-N row format (fv, bv, oa, ob)
struct TpArgs {
  int L;                        // chunk length (steps)
  const float* logb;            // [total_T][N] natural log
  const int64_t* offsets;
  const int32_t* model_id;
  ModelView mv;
  const int32_t* chunk_seq;     // [n_chunks] sequence of each chunk
  const int32_t* chunk_t0;      // [n_chunks] first step of each chunk
  const int32_t* seq_chunk0;    // [n_seq] first chunk of each sequence
  const int32_t* seq_nchunk;    // [n_seq] its chunk count
  float* Q;                     // [n_chunks][2][NP][NP] transfer matrices (rows scaled)
  long long* qexp;              // [n_chunks][2][NP] log2 row scales (integers)
  float* bvec;                  // [n_chunks][2][NP] boundary vectors
  long long* boff;              // [n_chunks][2] their log2 offsets (integers)
  float* fv;
  float* bv;
  double* oa;
  double* ob;
};
cudaError_t launch_tp_fb(int NP, const TpArgs& a, int n_chunks, int n_seq, cudaStream_t st);
// posterior rows: gamma [total_T][N], 1/Z_t [total_T], log-likelihoods
cudaError_t launch_large_post(const LargeArgs& a, int NP, int N, int64_t n_seq, int64_t max_T, float* gamma,
                              float* rz, double* loglik, int* status, cudaStream_t st);
// per-sequence statistic partials [n_seq][NP][NST] (slot NST-1: gamma_1)
cudaError_t launch_large_stats(const LargeArgs& a, const float* y, const float* gamma, int64_t n_seq, bool table,
                               float* part, cudaStream_t st);
// xi blocks per chunk [n_chunks][NP][NP] (float64, without the a_ij factor)
cudaError_t launch_large_xi(const LargeArgs& a, const float* rz, const int32_t* seq_by_model, const int32_t* chunk_lo,
                            const int32_t* chunk_hi, int n_chunks, double* xi_chunk, cudaStream_t st);
// chunk records in the rec_size(NP) layout
cudaError_t launch_large_reduce(const float* part, const double* loglik, const double* xi_chunk,
                                const int32_t* seq_by_model, const int32_t* chunk_lo, const int32_t* chunk_hi,
                                int n_chunks, int NP, double* chunk_rec, cudaStream_t st);

}  // namespace hmm
