// Host-side runtime objects of the hmmgpu library: error handling, the
// context workspace, device models and batch plans.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hmmgpu.h"
#include "common.cuh"
#include "mstep_types.h"

namespace hmm {

void set_error(const std::string& msg);

struct Error {
  hmm_status st;
  std::string msg;
};

#define HMM_CUDA(call)                                                                               \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      throw ::hmm::Error{HMM_E_CUDA, std::string(#call) + " (" + ::hmm::src_base(__FILE__) + ":" +     \
                                         std::to_string(__LINE__) + "): " + cudaGetErrorString(e_)}; \
  } while (0)

// file name without its directories (error messages)
inline const char* src_base(const char* f) {
  const char* b = f;
  for (const char* p = f; *p; ++p)
    if (*p == '/') b = p + 1;
  return b;
}

#define HMM_REQUIRE(cond, msg)                                            \
  do {                                                                    \
    if (!(cond)) throw ::hmm::Error{HMM_E_ARG, std::string(msg)};         \
  } while (0)

// Stream for stream-ordered allocation on this thread (nullptr: plain
// cudaMalloc / cudaFree).  The request server's slot threads set it to their
// stream, so that growing a buffer never waits for the other slots' work
// (cudaFree synchronises the whole device).
cudaStream_t& alloc_stream();

// A growable device buffer owned by the library.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t owner = nullptr;   // stream of a stream-ordered allocation
  void free_now() {
    if (!p) return;
    if (owner) {
      // stream-ordered memory is returned on the stream it was taken on
      cudaFreeAsync(p, owner);
    } else {
      cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    owner = nullptr;
  }
  void ensure(size_t n) {
    if (n <= bytes) return;
    free_now();
    cudaStream_t s = alloc_stream();
    cudaError_t e;
    if (s) {
      e = cudaMallocAsync(&p, n, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // usable from any stream
      owner = s;
    } else {
      e = cudaMalloc(&p, n);
    }
    if (e != cudaSuccess) {
      p = nullptr;
      owner = nullptr;
      throw Error{HMM_E_NOMEM, "cudaMalloc(" + std::to_string(n) + "): " + cudaGetErrorString(e)};
    }
    bytes = n;
  }
  void release() { free_now(); }
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

}  // namespace hmm

struct hmm_ctx_s {
  int device = 0;
  int n_sm = 0;
  int* status = nullptr;         // device status word
  int* counters = nullptr;       // device work counters [64]
  cudaStream_t work_stream = nullptr;  // non-blocking stream for captured loops
  hmm::DevBuf scratch;           // [total_T][NP] float recurrence rows
  hmm::DevBuf partials;          // per-sequence float32 partial sums
  hmm::DevBuf chunk_rec;         // float64 chunk records
  hmm::DevBuf loglik;            // float64 per-sequence logL (internal)
  hmm::DevBuf psi;               // Viterbi backpointers
  hmm::DevBuf gamma;             // gamma rows for the data passes
  hmm::DevBuf dp_part;           // data-pass partials
  hmm::DevBuf trace;             // float64 logL trace of hmm_fit
  hmm::DevBuf plain_beta;        // beta-hat rows of the plain path
  hmm::DevBuf tune_out;          // outputs of the autotuner's trial runs
  hmm::DevBuf mvlogb;            // [total_T][N] log b table (multivariate and large-N models)
  hmm::DevBuf lg_bv;             // [total_T][NP] large-N backward rows
  hmm::DevBuf lg_logAT;          // [M][NP][NP] ln a transposed (large-N Viterbi traceback)
  hmm::DevBuf lg_off;            // [2][total_T] float64 log2 offsets (forward, backward)
  hmm::DevBuf lg_rz;             // [total_T] 1 / Z_t
  hmm::DevBuf lg_xi;             // [n_chunks][NP][NP] float64 xi blocks
  hmm::DevBuf xi_xt, xi_yt;      // [NP][xi_ktot] float32 operands of the tensor-core xi
  hmm::DevBuf vt_path;           // [total_T] Viterbi paths of Viterbi training
  hmm::DevBuf vt_count;          // [n_chunks][NP][NP] int32 transition counts
  hmm::DevBuf km_u, km_d2, km_part, km_flags;   // k-means++: uniforms, D2, block sums, flags
  // options
  int profile = 0;
  int estep_lanes = 0;
  int viterbi_lanes = 0;
  int plain_estep = 0;
  int tensor_rec = 0;            // HMM_OPT_TENSOR_RECURRENCE
  int time_parallel = 0;         // HMM_OPT_TIME_PARALLEL
  hmm::DevBuf tp_Q, tp_qexp, tp_bvec, tp_boff;   // time-parallel chunk data
  // kernel timing
  struct Rec {
    int slot;
    cudaEvent_t e0, e1;
    int kernels;                 // kernels launched between e0 and e1
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> event_pool;
  double kt_ms[HMM_KT_SLOTS] = {0};
  int64_t kt_n[HMM_KT_SLOTS] = {0};
};

struct hmm_model_s {
  hmm_ctx ctx = nullptr;
  int M = 0, N = 0, NP = 0, D = 1, P = 0;
  std::vector<int32_t> h_family;
  bool any_negbin = false, any_weibull = false, any_mv = false, any_discrete = false;
  int K = 0;                     // symbols of the discrete family
  int dim_arg = 1;               // the `dim` the model was created with (K for discrete)
  hmm::DevBuf dtab;              // [M][NP][K] float32 ln p_jk (discrete family)
  // the last family group (log-normal .. Pareto): densities through the
  // table, statistics from the occupancies; uniform / Pareto also need the
  // support min / max
  bool any_ext = false, any_support = false;
  // independent components (HMM_INDEP): the component family of each
  // dimension per model, density coefficients [M][NP][D][KC] and shifts
  // [M][NP][D] per component
  bool any_indep = false;
  std::vector<int32_t> h_icomp;  // [M][D]
  hmm::DevBuf icomp, icoef, ishift;
  bool table_family() const { return any_mv || any_discrete || any_ext || any_indep; }
  hmm::DevBuf family, pi, A, theta, A32, AT32, logA2, logAe, pi32, logpi2, logpie, coef, nbtab, lfact2;
  int KM = 0, KS = 0;            // multivariate coefficient / statistic slots per state
  hmm::DevBuf mvcoef;            // [M][NP][KM] float32 (multivariate families)
  hmm::ModelBufs bufs() const;
  hmm::ModelView view() const;
};

struct hmm_stats_s {
  hmm_model model = nullptr;
  hmm::DevBuf rec;               // [M][rec_size(NP)] float64
  bool valid = false;
  // data-pass families (Weibull, negative binomial): occupancies of the last
  // E-step and the Newton state
  hmm::DevBuf gamma;             // [total_T][N] float32
  int64_t gamma_T = -1;          // total_T of the batch that wrote gamma
  hmm::DevBuf dps;               // [M][NP] DPState
  hmm::DevBuf dp_part;           // [S][NP][3] float32
  hmm::DevBuf dp_chunk;          // [n_chunks][NP*3] float64
  hmm::DevBuf dp_rec;            // [M][NP*3] float64
  hmm::DevBuf nb_hist;           // [M][NP][NB_YMAX] u64 fixed-point occupancy histograms
  hmm::DevBuf nb_tail;           // [S] u8: the sequence holds a count >= NB_YMAX
  hmm::DevBuf dp_count;          // active-state counters of the passes
  hmm::DevBuf mv_part;           // [S][NP][KS] float32 multivariate moments
  hmm::DevBuf mv_split;          // [n_chunks][split][NP][KS] float64 row-split partial moments
  hmm::DevBuf mv_chunk;          // [n_chunks][NP*KS] float64
  hmm::DevBuf mv_rec;            // [M][NP*KS] float64
  hmm::DevBuf ext_mm;            // [M][NP][2] int32 ordered keys of the support min / max
  bool hard = false;             // made by hmm_estep_viterbi: xi slots hold counts
  // cross-process exchange (hmm_stats_set_allreduce)
  hmm_allreduce_fn reduce_fn = nullptr;
  void* reduce_user = nullptr;
};

struct hmm_plan_s {
  hmm_ctx ctx = nullptr;
  int64_t n_seq = 0, total_T = 0;
  int M = 0;
  int64_t max_T = 0;
  hmm::DevBuf order;             // [S] int32 processing order
  hmm::DevBuf fam_seg_seq;       // [n_fam_seg + 1] family segments of the order (mixed-family batches)
  hmm::DevBuf fam_seg_sm;        // [n_fam_seg + 1] SM shares of the segments
  int n_fam_seg = 0;
  hmm::DevBuf seq_by_model;      // [S] int32
  hmm::DevBuf chunk_lo, chunk_hi;// [n_chunks] int32
  hmm::DevBuf model_chunk_ptr;   // [M+1] int32
  hmm::DevBuf chunk_row0;        // [S] int64: rows of the chunk's earlier sequences (seq_by_model order)
  int64_t max_chunk_rows = 0;    // rows of the longest chunk
  int n_chunks = 0;
  int uniform_family = -1;       // the one family of all sequences, or -1
  int estep_G = 0;               // chain widths chosen by hmm_plan_autotune (0: default)
  hmm::DevBuf tile_seq, tile_row;// 32-row tiles of the batch (multivariate emissions)
  int n_tiles = 0;
  hmm::DevBuf lg_groups;         // [n_groups][LG_SB] large-N sequence groups (one model each)
  int n_groups = 0;
  int lg_fill = 0;               // most sequences in one large-N group
  hmm::DevBuf tc_tiles;          // [n_tc_tiles][tc_tile_rows()] tiles of the tensor-core recursions
  int n_tc_tiles = 0;
  // chunk-ordered K layout of the tensor-core xi (padded N > 32): row t of
  // sequence s sits at K index xi_kseq[s] + t; chunk c covers
  // [xi_kc0[c], xi_kc0[c] + xi_kpad[c]) of which xi_kused[c] are rows
  hmm::DevBuf xi_kseq, xi_kc0, xi_kused, xi_kpad;
  int64_t xi_ktot = 0;
  // time-parallel chunks (padded N <= 32): chunk -> (sequence, first step),
  // sequence -> (first chunk, chunk count)
  hmm::DevBuf tp_chunk_seq, tp_chunk_t0, tp_seq_chunk0, tp_seq_nchunk;
  int n_tp_chunks = 0;
  int tp_L = 128;                // chunk length of the time-parallel path
  int viterbi_G = 0;
  std::vector<int32_t> h_order;
};

namespace hmm {
// Internal entry points shared by the C ABI and the request server.
// Fills (or refills) a plan for a batch from host offsets and model ids.
void fill_plan(hmm_plan p, hmm_ctx ctx, hmm_model model, const hmm_batch* b, const int64_t* ho, const int32_t* hm);
void destroy_plan(hmm_plan p);
// `iters` Baum-Welch iterations enqueued on `st` with no host
// synchronisation (stats and every scratch buffer must already be sized by
// one earlier E-step on this batch); returns the context-owned device trace
// [iters][M] of per-model log-likelihood sums.
const double* fit_async(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, hmm_stats stats,
                        const hmm_mstep_opts* opts, int iters, cudaStream_t st);
// Enqueues the E-step with statistics (used to size buffers before fit_async).
void estep_async(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, hmm_stats stats, double* d_loglik,
                 cudaStream_t st);
}  // namespace hmm
