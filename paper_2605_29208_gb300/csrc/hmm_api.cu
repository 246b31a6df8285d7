// Implementation of the hmmgpu C ABI (include/hmmgpu.h): contexts, models,
// plans, the inference entry points and the Baum-Welch loop.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "launch.h"
#include "mstep.cuh"
#include "mv.cuh"
#include "ext.cuh"
#include "indep.cuh"
#include "plain.cuh"
#include "runtime.h"

namespace hmm {

static thread_local std::string g_last_error;
cudaStream_t& alloc_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}
void set_error(const std::string& msg) { g_last_error = msg; }

template <class F>
static hmm_status guarded(F&& f) {
  try {
    f();
    return HMM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return HMM_E_ARG;
  } catch (...) {
    set_error("unknown exception");
    return HMM_E_ARG;
  }
}

static int padded_states(int N) {
  int np = 2;
  while (np < N) np *= 2;
  return np;
}

static int scalar_param_count(int fam) {
  switch (fam) {
    case HMM_GAUSS: return 2;
    case HMM_POISSON: return 1;
    case HMM_GAMMA: return 2;
    case HMM_BETA: return 2;
    case HMM_WEIBULL: return 2;
    case HMM_NEGBIN: return 2;
    case HMM_STUDENT_T: return 3;
    case HMM_VONMISES: return 2;
    case HMM_LOGNORMAL: return 2;
    case HMM_EXPONENTIAL: return 1;
    case HMM_RAYLEIGH: return 1;
    case HMM_UNIFORM: return 2;
    case HMM_CHISQ: return 1;
    case HMM_PARETO: return 2;
    default: return -1;
  }
}

static int param_count(int fam, int D) {
  if (fam == HMM_DISCRETE) return D;      // D = number of symbols
  if (fam == HMM_DIAG_GAUSS) return 2 * D;
  if (fam == HMM_FULL_GAUSS) return D + D * D;
  return scalar_param_count(fam);
}

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Parameters per state of model m (any family, independent components too).
static int model_param_count(hmm_model model, int m) {
  if (model->h_family[m] != HMM_INDEP) return param_count(model->h_family[m], model->dim_arg);
  int pc = 0;
  for (int d = 0; d < model->D; ++d) pc += indep_param_count(model->h_icomp[(size_t)m * model->D + d]);
  return pc;
}

static int64_t model_blob_size(hmm_model model) {
  int64_t tot = 0;
  const int64_t N = model->N;
  for (int m = 0; m < model->M; ++m) tot += N + N * N + N * model_param_count(model, m);
  return tot;
}

// Domain of one scalar family's parameters q (hmm_model_set_params).
static void check_scalar_params(int fam, const double* q) {
  switch (fam) {
    case HMM_LOGNORMAL: HMM_REQUIRE(q[1] > 0.0, "log-normal sigma2 must be > 0"); break;
    case HMM_EXPONENTIAL: HMM_REQUIRE(q[0] > 0.0, "exponential rate must be > 0"); break;
    case HMM_RAYLEIGH: HMM_REQUIRE(q[0] > 0.0, "Rayleigh sigma2 must be > 0"); break;
    case HMM_UNIFORM: HMM_REQUIRE(q[0] < q[1], "uniform bounds need a < b"); break;
    case HMM_CHISQ: HMM_REQUIRE(q[0] > 0.0, "chi-squared nu must be > 0"); break;
    case HMM_PARETO: HMM_REQUIRE(q[0] > 0.0 && q[1] > 0.0, "Pareto xm and alpha must be > 0"); break;
    default: break;
  }
}

// Records a pair of CUDA events around the launches made in its scope when
// the context's profiling option is on (not inside a graph capture).
// Grid of reduce_chunks_l2: one block row per model, the record's fields
// spread over blocks (each field is still one thread's fixed-order sum).
inline dim3 l2_grid(int M, int64_t RS, int threads) {
  const int64_t y = std::min<int64_t>(std::max<int64_t>((RS + threads - 1) / threads, 1), 4096);
  return dim3((unsigned)M, (unsigned)y);
}

struct KTimer {
  hmm_ctx ctx;
  int slot;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  int kernels = 1;             // kernels the region launches (set by the region)
  static cudaEvent_t take(hmm_ctx c) {
    if (!c->event_pool.empty()) {
      cudaEvent_t e = c->event_pool.back();
      c->event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  KTimer(hmm_ctx c, int sl, cudaStream_t s) : ctx(c), slot(sl), st(s) {
    if (!ctx || !ctx->profile) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    e0 = take(ctx);
    if (e0) cudaEventRecord(e0, st);
  }
  ~KTimer() {
    if (!e0) return;
    cudaEvent_t e1 = take(ctx);
    if (!e1) return;
    cudaEventRecord(e1, st);
    ctx->pending.push_back({slot, e0, e1, kernels});
  }
};

// ---------------------------------------------------------------- kernels
__global__ void post_path_kernel(const float* __restrict__ gamma, int64_t total_T, int N,
                                 int32_t* __restrict__ path) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_T) return;
  const float* g = gamma + t * N;
  float best = g[0];
  int arg = 0;
  for (int j = 1; j < N; ++j)
    if (g[j] > best) {
      best = g[j];
      arg = j;
    }
  path[t] = arg;
}

__global__ void trace_gather_kernel(const double* __restrict__ rec, int RS, int M,
                                    double* __restrict__ trace, int* __restrict__ it) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = *it;
  if (m < M) trace[(size_t)k * M + m] = rec[(size_t)m * RS + 1];
}

__global__ void bump_kernel(int* it) { *it += 1; }

// Single-state emission log-densities of a whole batch (natural log).
// Blocks (sequence, slab of EMIS_SLAB rows).
inline unsigned slabs_of(int64_t max_T) { return (unsigned)std::max<int64_t>(1, (max_T + EMIS_SLAB - 1) / EMIS_SLAB); }
__global__ void emission_kernel(ModelView mv, const float* __restrict__ y, const int64_t* __restrict__ offsets,
                                const int32_t* __restrict__ model_id, float* __restrict__ logb) {
  const int s = blockIdx.x;
  const int64_t b = offsets[s] + (int64_t)blockIdx.y * EMIS_SLAB;
  const int64_t e = min(offsets[s + 1], b + (int64_t)EMIS_SLAB);
  if (b >= e) return;
  const int m = model_id[s];
  const int fam = mv.family[m];
  const int N = mv.N, NP = mv.NP;
  if (N <= (int)blockDim.x) {
    // a fixed (row, state) slot per thread: blockDim / N rows per pass, the
    // state's coefficients in registers, stores coalesced along the row
    const int rpp = blockDim.x / N, rr = threadIdx.x / N, k = threadIdx.x % N;
    if (rr >= rpp) return;
    float c[KC];
#pragma unroll
    for (int z = 0; z < KC; ++z) c[z] = mv.coef[((size_t)m * NP + k) * KC + z];
    const float* nbt = mv.nbtab ? mv.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
    for (int64_t t = b + rr; t < e; t += rpp) {
      const Feat f = feat_of(fam, y[t], mv.lfact2);
      const float l2 = f.ok ? emis_log2(fam, f, c, nbt) : -INFINITY;
      logb[t * N + k] = l2 * kLn2f;
    }
    return;
  }
  for (int64_t idx = threadIdx.x; idx < (e - b) * N; idx += blockDim.x) {
    const int64_t t = b + idx / N;
    const int k = (int)(idx % N);
    const Feat f = feat_of(fam, y[t], mv.lfact2);
    const float* c = mv.coef + ((size_t)m * NP + k) * KC;
    const float* nbt = mv.nbtab ? mv.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
    const float l2 = f.ok ? emis_log2(fam, f, c, nbt) : -INFINITY;
    logb[t * N + k] = l2 * kLn2f;
  }
}

template <int NP>
cudaError_t launch_plain_np(const PlainArgs& a, cudaStream_t st) {
  const int spb = 4 * (32 / NP);
  const unsigned grid = (unsigned)((a.n_seq + spb - 1) / spb);
  plain_recursions_kernel<NP><<<grid, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  plain_posterior_kernel<NP><<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_plain(int NP, const PlainArgs& a, cudaStream_t st) {
  switch (NP) {
    case 2: return launch_plain_np<2>(a, st);
    case 4: return launch_plain_np<4>(a, st);
    case 8: return launch_plain_np<8>(a, st);
    case 16: return launch_plain_np<16>(a, st);
    case 32: return launch_plain_np<32>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hmm

using namespace hmm;

// ================================================================ model views
ModelBufs hmm_model_s::bufs() const {
  ModelBufs b;
  b.M = M;
  b.N = N;
  b.NP = NP;
  b.D = D;
  b.P = P;
  b.family = family.as<int>();
  b.pi = pi.as<double>();
  b.A = A.as<double>();
  b.theta = theta.as<double>();
  b.A32 = A32.as<float>();
  b.AT32 = NP > 32 ? AT32.as<float>() : nullptr;
  b.logA2 = logA2.as<float>();
  b.logAe = logAe.as<float>();
  b.pi32 = pi32.as<float>();
  b.logpi2 = logpi2.as<float>();
  b.logpie = logpie.as<float>();
  b.coef = coef.as<float>();
  b.nbtab = any_negbin ? nbtab.as<float>() : nullptr;
  b.lfact2 = lfact2.as<float>();
  return b;
}

ModelView hmm_model_s::view() const {
  ModelView v;
  v.M = M;
  v.N = N;
  v.NP = NP;
  v.D = D;
  v.family = family.as<int>();
  v.A32 = A32.as<float>();
  v.AT32 = NP > 32 ? AT32.as<float>() : nullptr;
  v.logA2 = logA2.as<float>();
  v.logAe = logAe.as<float>();
  v.pi32 = pi32.as<float>();
  v.logpi2 = logpi2.as<float>();
  v.logpie = logpie.as<float>();
  v.coef = coef.as<float>();
  v.nbtab = any_negbin ? nbtab.as<float>() : nullptr;
  v.lfact2 = lfact2.as<float>();
  return v;
}

// ================================================================ helpers
namespace {

void check_batch(hmm_model model, const hmm_batch* b) {
  HMM_REQUIRE(b != nullptr, "batch is NULL");
  HMM_REQUIRE(b->n_seq >= 0 && b->total_T >= 0, "negative batch sizes");
  HMM_REQUIRE(b->n_seq < (1ll << 31) && b->total_T < (1ll << 40), "batch too large");
  HMM_REQUIRE(b->offsets != nullptr && (b->n_seq == 0 || b->model_id != nullptr), "batch arrays are NULL");
  HMM_REQUIRE(b->total_T == 0 || b->values != nullptr, "batch values are NULL");
  HMM_REQUIRE(b->dim == model->D, "batch dim does not match the model");
}

}  // namespace

// Fills (or refills) a plan for the batch; device buffers only grow, so a
// plan reused for batches of similar size allocates nothing.
void hmm::fill_plan(hmm_plan p, hmm_ctx ctx, hmm_model model, const hmm_batch* b, const int64_t* ho,
                    const int32_t* hm) {
  const int64_t S = b->n_seq;
  HMM_REQUIRE(S == 0 || (ho && hm), "host offsets/model_id needed for a plan");
  if (S > 0) {
    HMM_REQUIRE(ho[0] == 0, "offsets[0] must be 0");
    HMM_REQUIRE(ho[S] == b->total_T, "offsets[n_seq] must equal total_T");
  }
  int64_t maxT = 0;
  for (int64_t s = 0; s < S; ++s) {
    HMM_REQUIRE(ho[s + 1] >= ho[s], "offsets must be non-decreasing");
    HMM_REQUIRE(ho[s + 1] - ho[s] < (1ll << 30), "sequence longer than 2^30");
    HMM_REQUIRE(hm[s] >= 0 && hm[s] < model->M, "model_id out of range");
    maxT = std::max(maxT, ho[s + 1] - ho[s]);
  }
  {
    p->ctx = ctx;
    p->n_tiles = 0;
    p->n_tp_chunks = 0;
    p->n_groups = 0;
    p->n_tc_tiles = 0;
    p->estep_G = 0;
    p->viterbi_G = 0;
    p->n_seq = S;
    p->total_T = b->total_T;
    p->M = model->M;
    p->max_T = maxT;
    std::vector<int32_t> order(S), bym(S);
    std::iota(order.begin(), order.end(), 0);
    std::iota(bym.begin(), bym.end(), 0);
    // Processing order: longest first in buckets of ~9% length (so that the
    // persistent warps take the long sequences early), family inside a
    // bucket (family-uniform warps), then exact length descending.  A batch
    // that mixes the fused families (one kernel holding every family's loop)
    // is laid out family first instead, one segment per family in that
    // order, and the kernels give each segment its own SMs (FamSched).
    auto bucket = [&](int32_t q) {
      const int64_t L = ho[q + 1] - ho[q];
      return L <= 0 ? -1 : (int)std::floor(8.0 * std::log2((double)L));
    };
    bool mixed = false;
    for (int64_t q2 = 1; q2 < S && !mixed; ++q2) mixed = model->h_family[hm[q2]] != model->h_family[hm[0]];
    const bool fam_major = mixed && model->NP <= 32 && !model->table_family();
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
      const int fx = model->h_family[hm[x]], fy = model->h_family[hm[y]];
      if (fam_major && fx != fy) return fx < fy;
      const int bx = bucket(x), by = bucket(y);
      if (bx != by) return bx > by;
      if (fx != fy) return fx < fy;
      return (ho[x + 1] - ho[x]) > (ho[y + 1] - ho[y]);
    });
    p->n_fam_seg = 0;
    if (fam_major) {
      std::vector<int32_t> sseq{0};
      std::vector<double> w;
      double wsum = 0.0;
      for (int64_t q2 = 0; q2 < S; ++q2) {
        if (q2 > 0 && model->h_family[hm[order[q2]]] != model->h_family[hm[order[q2 - 1]]]) {
          sseq.push_back((int32_t)q2);
          w.push_back(0.0);
        }
        if (w.empty()) w.push_back(0.0);
        const double L = (double)(ho[order[q2] + 1] - ho[order[q2]]);
        w.back() += L;
        wsum += L;
      }
      sseq.push_back((int32_t)S);
      const int nseg = (int)w.size();
      const int nsm = std::max(ctx->n_sm, 1);
      std::vector<int32_t> ssm(nseg + 1, 0);
      double cum = 0.0;
      for (int f = 0; f < nseg; ++f) {
        cum += w[f];
        ssm[f + 1] = f + 1 == nseg ? nsm : (int32_t)std::llround(nsm * (wsum > 0 ? cum / wsum : 1.0));
      }
      HMM_REQUIRE(nseg <= 8, "more than 8 family segments");
      p->n_fam_seg = nseg;
      p->fam_seg_seq.ensure((size_t)(nseg + 1) * 4);
      p->fam_seg_sm.ensure((size_t)(nseg + 1) * 4);
      HMM_CUDA(cudaMemcpy(p->fam_seg_seq.p, sseq.data(), (nseg + 1) * 4, cudaMemcpyHostToDevice));
      HMM_CUDA(cudaMemcpy(p->fam_seg_sm.p, ssm.data(), (nseg + 1) * 4, cudaMemcpyHostToDevice));
    }
    std::stable_sort(bym.begin(), bym.end(), [&](int32_t x, int32_t y) { return hm[x] < hm[y]; });
    const int CH = 64;
    std::vector<int32_t> lo, hi, mptr(model->M + 1, 0);
    int64_t q = 0;
    for (int m = 0; m < model->M; ++m) {
      mptr[m] = (int32_t)lo.size();
      int64_t e = q;
      while (e < S && hm[bym[e]] == m) ++e;
      for (int64_t c = q; c < e; c += CH) {
        lo.push_back((int32_t)c);
        hi.push_back((int32_t)std::min<int64_t>(c + CH, e));
      }
      q = e;
    }
    mptr[model->M] = (int32_t)lo.size();
    p->n_chunks = (int)lo.size();
    {
      std::vector<int64_t> crow(std::max<int64_t>(S, 1), 0);
      p->max_chunk_rows = 0;
      for (size_t c = 0; c < lo.size(); ++c) {
        int64_t acc = 0;
        for (int32_t q2 = lo[c]; q2 < hi[c]; ++q2) {
          crow[q2] = acc;
          acc += ho[bym[q2] + 1] - ho[bym[q2]];
        }
        p->max_chunk_rows = std::max(p->max_chunk_rows, acc);
      }
      p->chunk_row0.ensure(crow.size() * 8);
      HMM_CUDA(cudaMemcpy(p->chunk_row0.p, crow.data(), crow.size() * 8, cudaMemcpyHostToDevice));
    }
    p->order.ensure(std::max<int64_t>(S, 1) * 4);
    p->seq_by_model.ensure(std::max<int64_t>(S, 1) * 4);
    p->chunk_lo.ensure(std::max<size_t>(lo.size(), 1) * 4);
    p->chunk_hi.ensure(std::max<size_t>(lo.size(), 1) * 4);
    p->model_chunk_ptr.ensure(mptr.size() * 4);
    if (S) {
      HMM_CUDA(cudaMemcpy(p->order.p, order.data(), S * 4, cudaMemcpyHostToDevice));
      HMM_CUDA(cudaMemcpy(p->seq_by_model.p, bym.data(), S * 4, cudaMemcpyHostToDevice));
    }
    if (!lo.empty()) {
      HMM_CUDA(cudaMemcpy(p->chunk_lo.p, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice));
      HMM_CUDA(cudaMemcpy(p->chunk_hi.p, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice));
    }
    HMM_CUDA(cudaMemcpy(p->model_chunk_ptr.p, mptr.data(), mptr.size() * 4, cudaMemcpyHostToDevice));
    if ((model->any_mv || model->NP > 32) && S > 0) {
      std::vector<int32_t> ts, tr;
      for (int64_t q2 = 0; q2 < S; ++q2)
        for (int64_t r = 0; r < ho[q2 + 1] - ho[q2]; r += 32) {
          ts.push_back((int32_t)q2);
          tr.push_back((int32_t)r);
        }
      p->n_tiles = (int)ts.size();
      p->tile_seq.ensure(std::max<size_t>(ts.size(), 1) * 4);
      p->tile_row.ensure(std::max<size_t>(tr.size(), 1) * 4);
      if (!ts.empty()) {
        HMM_CUDA(cudaMemcpy(p->tile_seq.p, ts.data(), ts.size() * 4, cudaMemcpyHostToDevice));
        HMM_CUDA(cudaMemcpy(p->tile_row.p, tr.data(), tr.size() * 4, cudaMemcpyHostToDevice));
      }
    }
    if (model->NP > 32 && S > 0) {
      // K layout of the tensor-core xi: the chunks' rows (t < T - 1) one
      // after another, each chunk padded to a multiple of 32
      std::vector<int64_t> kseq(S, 0), kc0(lo.size());
      std::vector<int32_t> kused(lo.size()), kpad(lo.size());
      int64_t ktot = 0;
      for (size_t c = 0; c < lo.size(); ++c) {
        kc0[c] = ktot;
        int64_t used = 0;
        for (int32_t q2 = lo[c]; q2 < hi[c]; ++q2) {
          const int32_t sq = bym[q2];
          kseq[sq] = ktot + used;
          used += std::max<int64_t>(ho[sq + 1] - ho[sq] - 1, 0);
        }
        HMM_REQUIRE(used < (1ll << 31) - 64, "chunk too long for the xi layout");
        kused[c] = (int32_t)used;
        kpad[c] = (int32_t)((used + 31) / 32 * 32);
        ktot += kpad[c];
      }
      p->xi_ktot = std::max<int64_t>(ktot, 32);
      p->xi_kseq.ensure((size_t)S * 8);
      p->xi_kc0.ensure(std::max<size_t>(lo.size(), 1) * 8);
      p->xi_kused.ensure(std::max<size_t>(lo.size(), 1) * 4);
      p->xi_kpad.ensure(std::max<size_t>(lo.size(), 1) * 4);
      HMM_CUDA(cudaMemcpy(p->xi_kseq.p, kseq.data(), (size_t)S * 8, cudaMemcpyHostToDevice));
      if (!lo.empty()) {
        HMM_CUDA(cudaMemcpy(p->xi_kc0.p, kc0.data(), lo.size() * 8, cudaMemcpyHostToDevice));
        HMM_CUDA(cudaMemcpy(p->xi_kused.p, kused.data(), lo.size() * 4, cudaMemcpyHostToDevice));
        HMM_CUDA(cudaMemcpy(p->xi_kpad.p, kpad.data(), lo.size() * 4, cudaMemcpyHostToDevice));
      }
    }
    if (model->NP > 32 && S > 0) {
      // groups of LG_SB sequences of one model with similar lengths, the
      // groups holding the longest sequences first
      std::vector<int32_t> idx(S);
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
        if (hm[x] != hm[y]) return hm[x] < hm[y];
        return (ho[x + 1] - ho[x]) > (ho[y + 1] - ho[y]);
      });
      std::vector<std::vector<int32_t>> groups;
      for (int64_t q2 = 0; q2 < S;) {
        std::vector<int32_t> g(LG_SB, -1);
        const int mq = hm[idx[q2]];
        for (int c = 0; c < LG_SB && q2 < S && hm[idx[q2]] == mq; ++c) g[c] = idx[q2++];
        groups.push_back(std::move(g));
      }
      std::stable_sort(groups.begin(), groups.end(), [&](const std::vector<int32_t>& x, const std::vector<int32_t>& y) {
        return (ho[x[0] + 1] - ho[x[0]]) > (ho[y[0] + 1] - ho[y[0]]);
      });
      std::vector<int32_t> flat;
      for (auto& g : groups) flat.insert(flat.end(), g.begin(), g.end());
      p->n_groups = (int)groups.size();
      p->lg_fill = 0;
      for (auto& g : groups) {
        int f = 0;
        for (int32_t x : g) f += x >= 0;
        p->lg_fill = std::max(p->lg_fill, f);
      }
      p->lg_groups.ensure(flat.size() * 4);
      HMM_CUDA(cudaMemcpy(p->lg_groups.p, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice));
      if (tc_supported(model->NP)) {
        // tiles of the tensor-core recursions: tc_tile_rows() sequences of
        // one model, longest first (the first entry of a tile is valid)
        const int TR = tc_tile_rows();
        std::vector<int32_t> tiles;
        int nt = 0;
        for (int64_t q2 = 0; q2 < S;) {
          const int mq = hm[idx[q2]];
          std::vector<int32_t> g(TR, -1);
          for (int c = 0; c < TR && q2 < S && hm[idx[q2]] == mq; ++c) g[c] = idx[q2++];
          tiles.insert(tiles.end(), g.begin(), g.end());
          ++nt;
        }
        p->n_tc_tiles = nt;
        p->tc_tiles.ensure(tiles.size() * 4);
        HMM_CUDA(cudaMemcpy(p->tc_tiles.p, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice));
      }
    }
    if (model->NP <= 32 && S > 0) {
      // time-parallel chunks of L steps: the boundary walk costs ~T/L
      // sequential chunk steps and the chunks ~L sequential steps each, so L
      // ~ sqrt(T) (a power of two in [64, 4096]) balances the two
      int L = 64;
      while (L < 4096 && (double)L * L < 4.0 * (double)maxT) L *= 2;
      p->tp_L = L;
      const int TP_L = L;
      std::vector<int32_t> cs, ct, s0(S), sn(S);
      for (int64_t q2 = 0; q2 < S; ++q2) {
        const int64_t Tq = ho[q2 + 1] - ho[q2];
        s0[q2] = (int32_t)cs.size();
        for (int64_t t = 0; t < Tq; t += TP_L) {
          cs.push_back((int32_t)q2);
          ct.push_back((int32_t)t);
        }
        sn[q2] = (int32_t)cs.size() - s0[q2];
      }
      p->n_tp_chunks = (int)cs.size();
      p->tp_chunk_seq.ensure(std::max<size_t>(cs.size(), 1) * 4);
      p->tp_chunk_t0.ensure(std::max<size_t>(ct.size(), 1) * 4);
      p->tp_seq_chunk0.ensure((size_t)S * 4);
      p->tp_seq_nchunk.ensure((size_t)S * 4);
      if (!cs.empty()) {
        HMM_CUDA(cudaMemcpy(p->tp_chunk_seq.p, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice));
        HMM_CUDA(cudaMemcpy(p->tp_chunk_t0.p, ct.data(), ct.size() * 4, cudaMemcpyHostToDevice));
      }
      HMM_CUDA(cudaMemcpy(p->tp_seq_chunk0.p, s0.data(), (size_t)S * 4, cudaMemcpyHostToDevice));
      HMM_CUDA(cudaMemcpy(p->tp_seq_nchunk.p, sn.data(), (size_t)S * 4, cudaMemcpyHostToDevice));
    }
    int uf = -2;
    for (int64_t q2 = 0; q2 < S; ++q2) {
      const int f = model->h_family[hm[q2]];
      uf = (uf == -2 || uf == f) ? f : -1;
    }
    p->uniform_family = uf < 0 ? -1 : uf;
    p->h_order = std::move(order);
  }
}

void hmm::destroy_plan(hmm_plan p) {
  if (!p) return;
  p->order.release();
  p->seq_by_model.release();
  p->chunk_lo.release();
  p->chunk_hi.release();
  p->model_chunk_ptr.release();
  p->tile_seq.release();
  p->tile_row.release();
  p->lg_groups.release();
  p->tc_tiles.release();
  for (auto* bb : {&p->chunk_row0, &p->xi_kseq, &p->xi_kc0, &p->xi_kused, &p->xi_kpad, &p->tp_chunk_seq, &p->tp_chunk_t0,
                   &p->tp_seq_chunk0, &p->tp_seq_nchunk, &p->fam_seg_seq, &p->fam_seg_sm})
    bb->release();
  delete p;
}

namespace {

// Builds a plan from host arrays.
hmm_plan make_plan(hmm_ctx ctx, hmm_model model, const hmm_batch* b, const int64_t* ho, const int32_t* hm) {
  auto* p = new hmm_plan_s();
  try {
    fill_plan(p, ctx, model, b, ho, hm);
  } catch (...) {
    destroy_plan(p);
    throw;
  }
  return p;
}

// A plan for the batch: the caller's, or a temporary one built from host
// copies of offsets and model_id (synchronous).
struct PlanRef {
  hmm_plan p = nullptr;
  bool owned = false;
  ~PlanRef() {
    if (owned) destroy_plan(p);
  }
};

void get_plan(hmm_ctx ctx, hmm_model model, const hmm_batch* b, cudaStream_t st, PlanRef& ref) {
  if (b->plan) {
    HMM_REQUIRE(b->plan->n_seq == b->n_seq && b->plan->total_T == b->total_T && b->plan->M == model->M,
                "plan does not match the batch");
    ref.p = b->plan;
    ref.owned = false;
    return;
  }
  std::vector<int64_t> ho(b->n_seq + 1);
  std::vector<int32_t> hm(std::max<int64_t>(b->n_seq, 1));
  HMM_CUDA(cudaStreamSynchronize(st));
  HMM_CUDA(cudaMemcpy(ho.data(), b->offsets, (b->n_seq + 1) * 8, cudaMemcpyDeviceToHost));
  if (b->n_seq) HMM_CUDA(cudaMemcpy(hm.data(), b->model_id, b->n_seq * 4, cudaMemcpyDeviceToHost));
  ref.p = make_plan(ctx, model, b, ho.data(), hm.data());
  ref.owned = true;
}

// Multivariate emission table: the tiled kernel when the model set has one
// multivariate family it covers, else the generic kernel.
void launch_mv_emission(hmm_model model, const hmm_batch* b, hmm_plan plan, float* out, cudaStream_t st) {
  int fam = model->h_family[0];
  for (int f : model->h_family)
    if (f != fam) fam = -1;
  const int D = model->D;
  if (fam == HMM_DIAG_GAUSS || (fam == HMM_FULL_GAUSS && D <= MV_TILED_FULL_D)) {
    const dim3 grid((unsigned)plan->n_tiles, (unsigned)((model->N + 63) / 64));
    const size_t smem = ((size_t)32 * (D + 1) + (size_t)64 * (model->KM | 1)) * 4;
    if (fam == HMM_DIAG_GAUSS) {
      auto kern = mv_emission_tiled_kernel<HMM_DIAG_GAUSS>;
      HMM_CUDA(ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem));
      kern<<<grid, 256, smem, st>>>(model->mvcoef.as<float>(), model->NP, model->N, D, model->KM, b->values,
                                    b->offsets, b->model_id, plan->tile_seq.as<int32_t>(),
                                    plan->tile_row.as<int32_t>(), out);
    } else {
      auto kern = mv_emission_tiled_kernel<HMM_FULL_GAUSS>;
      HMM_CUDA(ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem));
      kern<<<grid, 256, smem, st>>>(model->mvcoef.as<float>(), model->NP, model->N, D, model->KM, b->values,
                                    b->offsets, b->model_id, plan->tile_seq.as<int32_t>(),
                                    plan->tile_row.as<int32_t>(), out);
    }
  } else {
    mv_emission_kernel<<<(unsigned)plan->n_tiles, 128, (size_t)32 * D * 4, st>>>(
        model->family.as<int>(), model->mvcoef.as<float>(), model->NP, model->N, D, model->KM, b->values, b->offsets,
        b->model_id, plan->tile_seq.as<int32_t>(), plan->tile_row.as<int32_t>(), out);
  }
  HMM_CUDA(cudaGetLastError());
}

// log b table of the batch in the context's buffer: multivariate families
// (Sec. 4.5) one block per 32-row tile of a sequence, scalar families one
// block per sequence.
void launch_indep_emission(hmm_model model, const hmm_batch* b, hmm_plan plan, float* out, cudaStream_t st) {
  if (b->n_seq == 0) return;
  indep_emission_kernel<<<dim3((unsigned)b->n_seq, slabs_of(plan->max_T)), 128, 0, st>>>(
      model->icomp.as<int>(), model->icoef.as<float>(), model->NP, model->N, model->D, model->lfact2.as<float>(),
      b->values, b->offsets, b->model_id, out);
  HMM_CUDA(cudaGetLastError());
}

const float* mv_table(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, cudaStream_t st) {
  ctx->mvlogb.ensure(std::max<int64_t>(b->total_T, 1) * model->N * 4);
  if (model->any_indep) {
    KTimer kt(ctx, HMM_KT_EMISSION, st);
    launch_indep_emission(model, b, plan, ctx->mvlogb.as<float>(), st);
  } else if (model->any_discrete) {
    if (b->n_seq > 0) {
      KTimer kt(ctx, HMM_KT_EMISSION, st);
      discrete_emission_kernel<<<dim3((unsigned)b->n_seq, slabs_of(plan->max_T)), 128, 0, st>>>(
          model->dtab.as<float>(), model->NP, model->N, model->K, b->values, b->offsets, b->model_id,
          ctx->mvlogb.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
  } else if (!model->any_mv) {
    if (b->n_seq > 0) {
      KTimer kt(ctx, HMM_KT_EMISSION, st);
      emission_kernel<<<dim3((unsigned)b->n_seq, slabs_of(plan->max_T)), 128, 0, st>>>(
          model->view(), b->values, b->offsets, b->model_id, ctx->mvlogb.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
  } else if (plan->n_tiles > 0) {
    KTimer kt(ctx, HMM_KT_EMISSION, st);
    launch_mv_emission(model, b, plan, ctx->mvlogb.as<float>(), st);
  }
  return ctx->mvlogb.as<float>();
}

// Shifted weighted moments of the multivariate families from the
// occupancies in stats->gamma, reduced in fixed order into stats->mv_rec.
int mv_statistics(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, hmm_stats stats,
                  cudaStream_t st) {
  const int NP = model->NP, KS = model->KS, RS = NP * KS;
  const int64_t S = b->n_seq;
  if (model->any_indep) {   // per-component weighted sums, fixed-order reductions
    stats->mv_part.ensure((size_t)std::max<int64_t>(S, 1) * RS * 4);
    stats->mv_chunk.ensure((size_t)std::max(plan->n_chunks, 1) * RS * 8);
    stats->mv_rec.ensure((size_t)model->M * RS * 8);
    int nk = 1;
    if (S > 0) {
      indep_stats_kernel<<<(unsigned)S, 256, 0, st>>>(model->icomp.as<int>(), model->ishift.as<float>(),
                                                      model->theta.as<double>(), NP, model->N, model->D, model->P, KS,
                                                      b->values, stats->gamma.as<float>(), b->offsets, b->model_id,
                                                      stats->mv_part.as<float>());
      HMM_CUDA(cudaGetLastError());
      ++nk;
    }
    if (plan->n_chunks > 0) {
      reduce_records_l1<<<plan->n_chunks, 128, 0, st>>>(stats->mv_part.as<float>(), RS,
                                                      plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(),
                                                      plan->chunk_hi.as<int32_t>(), stats->mv_chunk.as<double>());
      HMM_CUDA(cudaGetLastError());
      ++nk;
    }
    reduce_chunks_l2<<<l2_grid(model->M, RS, 128), 128, 0, st>>>(stats->mv_chunk.as<double>(),
                                                                 plan->model_chunk_ptr.as<int32_t>(), RS,
                                               stats->mv_rec.as<double>());
    HMM_CUDA(cudaGetLastError());
    return nk;
  }
  const bool raw = model->any_discrete || model->any_ext;   // feature sums, no shift
  // few raw features at small N: per-sequence sums (feat_stats_kernel)
  const bool raw_small = raw && NP <= 32 && KS <= FEAT_SMALL_MAX;
  if (NP <= 32 && (!raw || raw_small)) stats->mv_part.ensure((size_t)std::max<int64_t>(S, 1) * RS * 4);
  stats->mv_chunk.ensure((size_t)std::max(plan->n_chunks, 1) * RS * 8);
  stats->mv_rec.ensure((size_t)model->M * RS * 8);
  (void)ctx;   // timed inside the caller's reduction region
  int nk = 0;
  if (raw_small) {
    if (S > 0) {
      feat_stats_kernel<<<(unsigned)S, 256, 0, st>>>(model->family.as<int>(), NP, model->N, KS, b->values,
                                                    stats->gamma.as<float>(), b->offsets, b->model_id,
                                                    stats->mv_part.as<float>());
      HMM_CUDA(cudaGetLastError());
      ++nk;
    }
    if (plan->n_chunks > 0) {
      reduce_records_l1<<<plan->n_chunks, 128, 0, st>>>(stats->mv_part.as<float>(), RS,
                                                      plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(),
                                                      plan->chunk_hi.as<int32_t>(), stats->mv_chunk.as<double>());
      HMM_CUDA(cudaGetLastError());
      ++nk;
    }
    reduce_chunks_l2<<<l2_grid(model->M, RS, 128), 128, 0, st>>>(stats->mv_chunk.as<double>(),
                                                                 plan->model_chunk_ptr.as<int32_t>(), RS,
                                               stats->mv_rec.as<double>());
    HMM_CUDA(cudaGetLastError());
    ++nk;
  }
  if (!raw_small && (NP > 32 || raw)) {
    // tiled raw moments per chunk (symbol counts for the discrete family),
    // fixed-order model sums, then the shift to the current means
    if (plan->n_chunks > 0) {
      // row splits of about 4096 rows (at most 64) so that long chunks run on
      // many blocks
      const int ftiles = (KS + MVM_TILE - 1) / MVM_TILE;
      const int split = (int)std::min<int64_t>(64, std::max<int64_t>(1, (plan->max_chunk_rows + 4095) / 4096));
      stats->mv_split.ensure((size_t)plan->n_chunks * split * RS * 8);
      mv_moments_kernel<<<dim3((unsigned)(((NP + MVM_TILE - 1) / MVM_TILE) * ftiles), (unsigned)plan->n_chunks,
                               (unsigned)split),
                          256, 0, st>>>(model->family.as<int>(), NP, model->N, model->D, KS, b->values,
                                        stats->gamma.as<float>(), b->offsets, b->model_id,
                                        plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(),
                                        plan->chunk_hi.as<int32_t>(), plan->chunk_row0.as<int64_t>(), split,
                                        stats->mv_split.as<double>());
      HMM_CUDA(cudaGetLastError());
      mv_split_combine_kernel<<<dim3((unsigned)std::min<int64_t>((RS + 255) / 256, 64), (unsigned)plan->n_chunks), 256,
                                0, st>>>(stats->mv_split.as<double>(), split, RS, stats->mv_chunk.as<double>());
      HMM_CUDA(cudaGetLastError());
    }
    reduce_chunks_l2<<<l2_grid(model->M, RS, 128), 128, 0, st>>>(stats->mv_chunk.as<double>(),
                                                                 plan->model_chunk_ptr.as<int32_t>(), RS,
                                               stats->mv_rec.as<double>());
    HMM_CUDA(cudaGetLastError());
    nk = 2 * (plan->n_chunks > 0) + 1;
  }
  if (raw) {   // counts and feature sums need no shift
    if (model->any_support) {   // support min / max of the uniform and Pareto states
        const int n = model->M * NP;
        stats->ext_mm.ensure((size_t)n * 2 * 4);
        ext_support_init_kernel<<<(n + 127) / 128, 128, 0, st>>>(stats->ext_mm.as<int>(), n);
        HMM_CUDA(cudaGetLastError());
        nk += 1;
        if (S > 0) {
          ext_support_kernel<<<dim3((unsigned)S, slabs_of(plan->max_T)), 128, (size_t)model->N * 2 * 4, st>>>(
              model->family.as<int>(), model->coef.as<float>(), NP, model->N, b->values, b->offsets, b->model_id,
              stats->ext_mm.as<int>());
          HMM_CUDA(cudaGetLastError());
          nk += 1;
        }
    }
    return nk;
  }
  if (NP > 32) {
    const int n = model->M * NP;
    mv_shift_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->family.as<int>(), model->mvcoef.as<float>(), model->M,
                                                     NP, model->N, model->D, model->KM, KS,
                                                     stats->mv_rec.as<double>());
    HMM_CUDA(cudaGetLastError());
    return 2 * (plan->n_chunks > 0) + 2;
  }
  if (S > 0) {
    mv_stats_kernel<<<(unsigned)S, 128, 0, st>>>(model->family.as<int>(), model->mvcoef.as<float>(), NP, model->N,
                                                 model->D, model->KM, KS, b->values, stats->gamma.as<float>(),
                                                 b->offsets, b->model_id, stats->mv_part.as<float>());
    HMM_CUDA(cudaGetLastError());
  }
  if (plan->n_chunks > 0) {
    reduce_records_l1<<<plan->n_chunks, 128, 0, st>>>(stats->mv_part.as<float>(), RS, plan->seq_by_model.as<int32_t>(),
                                                    plan->chunk_lo.as<int32_t>(), plan->chunk_hi.as<int32_t>(),
                                                    stats->mv_chunk.as<double>());
    HMM_CUDA(cudaGetLastError());
  }
  reduce_chunks_l2<<<l2_grid(model->M, RS, 128), 128, 0, st>>>(stats->mv_chunk.as<double>(),
                                                                 plan->model_chunk_ptr.as<int32_t>(), RS,
                                             stats->mv_rec.as<double>());
  HMM_CUDA(cudaGetLastError());
  return (S > 0) + (plan->n_chunks > 0) + 1;
}

// Large-N E-step (padded N > 32): emission table, forward and backward
// recursions, posterior rows, then (for statistics) the per-sequence sums,
// the xi blocks and the fixed-order reductions.
void run_estep_large(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, const float* logb,
                     float* gamma, double* ll, bool want_stats, hmm_stats stats, cudaStream_t st) {
  const int NP = model->NP, N = model->N;
  const int64_t S = b->n_seq, TT = std::max<int64_t>(b->total_T, 1);
  if (want_stats && stats) stats->hard = false;
  if (ctx->plain_estep) throw Error{HMM_E_UNSUPPORTED, "the plain path covers padded N <= 32"};
  if (!logb) logb = mv_table(ctx, model, b, plan, st);
  ctx->scratch.ensure(TT * NP * 4 + 64);
  ctx->lg_bv.ensure(TT * NP * 4);
  ctx->lg_off.ensure(TT * 2 * 8);
  ctx->lg_rz.ensure(TT * 4);
  if (!gamma) {
    if (want_stats && stats) {
      stats->gamma.ensure(TT * N * 4);
      stats->gamma_T = b->total_T;
      gamma = stats->gamma.as<float>();
    } else {
      ctx->gamma.ensure(TT * N * 4);
      gamma = ctx->gamma.as<float>();
    }
  } else if (want_stats && stats && (model->table_family() || model->any_negbin || model->any_weibull)) {
    throw Error{HMM_E_ARG, "statistics of these families keep their own occupancies"};
  }
  if (want_stats) {
    ctx->partials.ensure((size_t)std::max<int64_t>(S, 1) * NP * NST * 4);
    ctx->lg_xi.ensure((size_t)std::max(plan->n_chunks, 1) * NP * NP * 8);
    ctx->chunk_rec.ensure((size_t)std::max(plan->n_chunks, 1) * rec_size(NP) * 8);
  }
  if (S == 0) return;
  LargeArgs a{};
  a.logb = logb;
  a.offsets = b->offsets;
  a.model_id = b->model_id;
  a.groups = plan->lg_groups.as<int32_t>();
  a.n_groups = plan->n_groups;
  a.group_fill = plan->lg_fill;
  a.status = ctx->status;
  a.mv = model->view();
  a.fv = ctx->scratch.as<float>();
  a.bv = ctx->lg_bv.as<float>();
  a.oa = ctx->lg_off.as<double>();
  a.ob = ctx->lg_off.as<double>() + TT;
  {
    KTimer kt(ctx, HMM_KT_ESTEP, st);
    if (ctx->tensor_rec && tc_supported(NP))
      HMM_CUDA(launch_tc_fb(NP, a, plan->tc_tiles.as<int32_t>(), plan->n_tc_tiles, ctx->status,
                            ctx->tensor_rec == 2 && tc_tf32_supported(NP), st));
    else
      HMM_CUDA(launch_large_fb(NP, a, st));
  }
  KTimer kt(ctx, HMM_KT_REDUCE, st);
  HMM_CUDA(launch_large_post(a, NP, N, S, plan->max_T, gamma, ctx->lg_rz.as<float>(), ll, ctx->status, st));
  if (!want_stats) return;
  kt.kernels = 4;   // post, statistics, xi reduction, model reduction (+ below)
  const bool table_stats = model->table_family();
  HMM_CUDA(launch_large_stats(a, b->values, gamma, S, table_stats, ctx->partials.as<float>(), st));
  if (ctx->tensor_rec && tc_xi_supported(NP)) {
    kt.kernels += 2 + (plan->n_tiles > 0);   // prep (+ pad) + GEMM in place of the CUDA-core xi
    ctx->xi_xt.ensure((size_t)NP * plan->xi_ktot * 4);
    ctx->xi_yt.ensure((size_t)NP * plan->xi_ktot * 4);
    KTimer kx(ctx, HMM_KT_XI, st);
    kx.kernels = 2 + (plan->n_tiles > 0);
    HMM_CUDA(launch_tc_xi(a, ctx->lg_rz.as<float>(), plan->tile_seq.as<int32_t>(), plan->tile_row.as<int32_t>(),
                          plan->n_tiles, plan->xi_kseq.as<int64_t>(), plan->xi_kc0.as<int64_t>(),
                          plan->xi_kused.as<int32_t>(), plan->xi_kpad.as<int32_t>(), plan->n_chunks, plan->xi_ktot,
                          ctx->xi_xt.as<float>(), ctx->xi_yt.as<float>(), ctx->lg_xi.as<double>(), ctx->status, st));
  } else {
    HMM_CUDA(launch_large_xi(a, ctx->lg_rz.as<float>(), plan->seq_by_model.as<int32_t>(),
                             plan->chunk_lo.as<int32_t>(), plan->chunk_hi.as<int32_t>(), plan->n_chunks,
                             ctx->lg_xi.as<double>(), st));
  }
  HMM_CUDA(launch_large_reduce(ctx->partials.as<float>(), ll, ctx->lg_xi.as<double>(),
                               plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(),
                               plan->chunk_hi.as<int32_t>(), plan->n_chunks, NP, ctx->chunk_rec.as<double>(), st));
  reduce_chunks_l2<<<l2_grid(model->M, rec_size(NP), 256), 256, 0, st>>>(ctx->chunk_rec.as<double>(),
                                                                         plan->model_chunk_ptr.as<int32_t>(),
                                             rec_size(NP), stats->rec.as<double>());
  HMM_CUDA(cudaGetLastError());
  kt.kernels += 1;   // the xi kernel of either form
  if (model->table_family()) kt.kernels += mv_statistics(ctx, model, b, plan, stats, st);
  stats->valid = true;
}

// Time-parallel forward-backward (no statistics) at padded N <= 32: the
// chunked transfer / boundary / recompute kernels write the rows of the
// large-N path and its posterior kernel finishes (gamma, log-likelihoods).
bool use_time_parallel(hmm_ctx ctx, hmm_model model, hmm_plan plan, bool want_stats) {
  if (want_stats || model->NP > 32 || ctx->time_parallel < 0 || ctx->plain_estep) return false;
  if (plan->n_tp_chunks == 0) return false;
  if (ctx->time_parallel > 0) return true;
  return plan->n_seq <= ctx->n_sm && plan->max_T >= 2048;
}

void run_fb_time_parallel(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, const float* logb,
                          float* gamma, double* ll, cudaStream_t st) {
  const int NP = model->NP, N = model->N;
  const int64_t S = b->n_seq, TT = std::max<int64_t>(b->total_T, 1);
  if (!logb) logb = mv_table(ctx, model, b, plan, st);
  ctx->scratch.ensure(TT * NP * 4 + 64);
  ctx->lg_bv.ensure(TT * NP * 4);
  ctx->lg_off.ensure(TT * 2 * 8);
  ctx->lg_rz.ensure(TT * 4);
  const size_t nc = (size_t)std::max(plan->n_tp_chunks, 1);
  ctx->tp_Q.ensure(nc * 2 * NP * NP * 4);
  ctx->tp_qexp.ensure(nc * 2 * NP * 8);
  ctx->tp_bvec.ensure(nc * 2 * NP * 4);
  ctx->tp_boff.ensure(nc * 2 * 8);
  if (!gamma) {
    ctx->gamma.ensure(TT * N * 4);
    gamma = ctx->gamma.as<float>();
  }
  if (S == 0) return;
  TpArgs t{};
  t.L = plan->tp_L;
  t.logb = logb;
  t.offsets = b->offsets;
  t.model_id = b->model_id;
  t.mv = model->view();
  t.chunk_seq = plan->tp_chunk_seq.as<int32_t>();
  t.chunk_t0 = plan->tp_chunk_t0.as<int32_t>();
  t.seq_chunk0 = plan->tp_seq_chunk0.as<int32_t>();
  t.seq_nchunk = plan->tp_seq_nchunk.as<int32_t>();
  t.Q = ctx->tp_Q.as<float>();
  t.qexp = ctx->tp_qexp.as<long long>();
  t.bvec = ctx->tp_bvec.as<float>();
  t.boff = ctx->tp_boff.as<long long>();
  t.fv = ctx->scratch.as<float>();
  t.bv = ctx->lg_bv.as<float>();
  t.oa = ctx->lg_off.as<double>();
  t.ob = ctx->lg_off.as<double>() + TT;
  {
    KTimer kt(ctx, HMM_KT_ESTEP, st);
    kt.kernels = 3;
    HMM_CUDA(launch_tp_fb(NP, t, plan->n_tp_chunks, (int)S, st));
  }
  LargeArgs a{};
  a.offsets = b->offsets;
  a.fv = t.fv;
  a.bv = t.bv;
  a.oa = t.oa;
  a.ob = t.ob;
  KTimer kt(ctx, HMM_KT_REDUCE, st);
  HMM_CUDA(launch_large_post(a, NP, N, S, plan->max_T, gamma, ctx->lg_rz.as<float>(), ll, ctx->status, st));
}

// The fused E-step over a batch.  gamma (optional) receives [total_T][N].
void run_estep(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, const float* logb,
               float* gamma, double* loglik, bool want_stats, hmm_stats stats, cudaStream_t st) {
  const int NP = model->NP;
  if (model->NP > 32) {
    double* ll = loglik;
    if (!ll) {
      ctx->loglik.ensure(std::max<int64_t>(b->n_seq, 1) * 8);
      ll = ctx->loglik.as<double>();
    }
    run_estep_large(ctx, model, b, plan, logb, gamma, ll, want_stats, stats, st);
    return;
  }
  if (use_time_parallel(ctx, model, plan, want_stats)) {
    double* ll = loglik;
    if (!ll) {
      ctx->loglik.ensure(std::max<int64_t>(b->n_seq, 1) * 8);
      ll = ctx->loglik.as<double>();
    }
    run_fb_time_parallel(ctx, model, b, plan, logb, gamma, ll, st);
    return;
  }
  if (model->table_family() && ctx->plain_estep)
    throw Error{HMM_E_UNSUPPORTED, "the plain path covers the scalar families only"};
  const int64_t S = b->n_seq;
  if (want_stats && stats) stats->hard = false;
  const bool mv_stats = want_stats && stats && model->table_family();
  if (model->table_family() && !logb) logb = mv_table(ctx, model, b, plan, st);
  ctx->scratch.ensure(std::max<int64_t>(b->total_T, 1) * NP * 4 + 64);
  const int F = NP + NST;
  ctx->partials.ensure(std::max<int64_t>(S, 1) * 2 * NP * F * 4);
  double* ll = loglik;
  if (!ll) {
    ctx->loglik.ensure(std::max<int64_t>(S, 1) * 8);
    ll = ctx->loglik.as<double>();
  }
  if (S == 0) return;
  if (ctx->plain_estep) {
    if (logb || gamma)
      throw Error{HMM_E_UNSUPPORTED, "the plain path computes log-likelihoods and statistics only"};
    ctx->plain_beta.ensure(std::max<int64_t>(b->total_T, 1) * NP * 4 + 64);
    PlainArgs pa;
    pa.y = b->values;
    pa.offsets = b->offsets;
    pa.model_id = b->model_id;
    pa.n_seq = (int32_t)S;
    pa.mv = model->view();
    pa.alpha = ctx->scratch.as<float>();
    pa.beta = ctx->plain_beta.as<float>();
    pa.partials = ctx->partials.as<float>();
    pa.loglik = ll;
    pa.gamma = nullptr;
    if (want_stats && stats && (model->any_negbin || model->any_weibull)) {
      // the data-pass M-steps re-read the occupancies of this E-step
      stats->gamma.ensure(std::max<int64_t>(b->total_T, 1) * model->N * 4);
      stats->gamma_T = b->total_T;
      pa.gamma = stats->gamma.as<float>();
    }
    {
      KTimer kt(ctx, HMM_KT_PLAIN, st);
      kt.kernels = 2;
      HMM_CUDA(launch_plain(NP, pa, st));
    }
  }
  EStepArgs a;
  a.y = b->values;
  a.logb = logb;
  a.offsets = b->offsets;
  a.model_id = b->model_id;
  a.order = plan->order.as<int32_t>();
  a.n_seq = (int32_t)S;
  int G = plan->estep_G > 0 ? plan->estep_G : default_estep_G(NP, S, ctx->n_sm);
  if (ctx->estep_lanes && estep_small_supported(NP, ctx->estep_lanes)) G = ctx->estep_lanes;
  a.n_items = (int32_t)((S + estep_seqs_per_item(G) - 1) / estep_seqs_per_item(G));
  a.mv = model->view();
  a.scratch = ctx->scratch.as<float>();
  a.gamma = gamma;
  a.partials = ctx->partials.as<float>();
  a.loglik = ll;
  a.work_counter = ctx->counters;
  a.status = ctx->status;
  if (plan->n_fam_seg > 0) {
    a.sched.n_seg = plan->n_fam_seg;
    a.sched.seg_seq = plan->fam_seg_seq.as<int32_t>();
    a.sched.seg_sm = plan->fam_seg_sm.as<int32_t>();
    a.work_counter = ctx->counters + 8;
  }
  const bool dpass = want_stats && stats && (model->any_negbin || model->any_weibull || model->table_family());
  if (dpass && !gamma) {
    // the Weibull / negative-binomial M-steps re-read the occupancies, and
    // the multivariate moments are formed from them
    stats->gamma.ensure(std::max<int64_t>(b->total_T, 1) * model->N * 4);
    stats->gamma_T = b->total_T;
    gamma = stats->gamma.as<float>();
    a.gamma = gamma;
  }
  if (!ctx->plain_estep) {
    HMM_CUDA(cudaMemsetAsync(a.work_counter, 0, sizeof(int) * std::max(a.sched.n_seg, 1), st));
    KTimer kt(ctx, HMM_KT_ESTEP, st);
    const int mode = (want_stats ? MODE_STATS : 0) | (gamma ? MODE_GAMMA : 0);
    const int fam = logb ? FAM_TABLE : (plan->uniform_family >= 0 ? plan->uniform_family : FAM_ANY);
    HMM_CUDA(launch_estep_small(NP, G, mode, a, fam, ctx->n_sm, st));
  }
  if (want_stats) {
    KTimer kt(ctx, HMM_KT_REDUCE, st);
    kt.kernels = (plan->n_chunks > 0) + 1;
    const int RS = rec_size(NP);
    ctx->chunk_rec.ensure((size_t)std::max(plan->n_chunks, 1) * RS * 8);
    if (plan->n_chunks > 0) {
      reduce_estep_l1<<<dim3((unsigned)plan->n_chunks, (unsigned)((RS + 127) / 128)), 128, 0, st>>>(
          a.partials, ll, plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(),
          plan->chunk_hi.as<int32_t>(), NP, ctx->chunk_rec.as<double>());
      HMM_CUDA(cudaGetLastError());
    }
    reduce_chunks_l2<<<l2_grid(model->M, RS, 128), 128, 0, st>>>(
        ctx->chunk_rec.as<double>(), plan->model_chunk_ptr.as<int32_t>(), RS, stats->rec.as<double>());
    HMM_CUDA(cudaGetLastError());
    if (mv_stats) kt.kernels += mv_statistics(ctx, model, b, plan, stats, st);
    stats->valid = true;
  }
}

MStepOpts to_opts(const hmm_mstep_opts* o) {
  MStepOpts r;
  r.collapse_eps = (o && o->collapse_eps > 0) ? o->collapse_eps : 1e-8;
  r.tikhonov_eps = (o && o->tikhonov_eps > 0) ? o->tikhonov_eps : 1e-6;
  r.newton_maxit = (o && o->newton_maxit > 0) ? o->newton_maxit : 50;
  r.newton_tol = (o && o->newton_tol > 0) ? o->newton_tol : 1e-10;
  r.nu_mode = o ? o->nu_mode : 0;
  r.update_transitions = o ? o->update_transitions : 1;
  r.prior_A = o ? o->dirichlet_A : 0.0;
  r.prior_pi = o ? o->dirichlet_pi : 0.0;
  r.hard = 0;
  return r;
}

// Buffers of the data-pass M-step (allocated before any graph capture).
// The caller's all-reduce on one device record (no-op without one).
void call_reduce(hmm_stats stats, void* p, int64_t n, int op, cudaStream_t st) {
  if (!stats->reduce_fn || n <= 0) return;
  const int32_t rc = stats->reduce_fn(p, n, op, reinterpret_cast<void*>(st), stats->reduce_user);
  if (rc != 0) throw Error{HMM_E_CUDA, "the all-reduce callback failed with code " + std::to_string(rc)};
}

// Record `index` of hmm_stats_record.
void record_view(hmm_stats stats, int index, void** p, int64_t* n, int* op) {
  hmm_model model = stats->model;
  const int64_t MNP = (int64_t)model->M * model->NP;
  switch (index) {
    case 0:
      *p = stats->rec.p;
      *n = (int64_t)model->M * rec_size(model->NP);
      *op = HMM_REDUCE_SUM_F64;
      return;
    case 1:
      *p = stats->mv_rec.p;
      *n = model->table_family() && stats->mv_rec.p ? MNP * model->KS : 0;
      *op = HMM_REDUCE_SUM_F64;
      return;
    case 2:
      *p = stats->ext_mm.p;
      *n = model->any_support && stats->ext_mm.p ? MNP * 2 : 0;
      *op = HMM_REDUCE_MIN_I32;
      return;
    default: throw Error{HMM_E_ARG, "record index must be 0, 1 or 2"};
  }
}

// Statistics of an empty shard: zero sums, the identity of the support
// minimum; valid for an M-step once combined with the other shards.
void zero_stats(hmm_model model, hmm_stats stats, cudaStream_t st) {
  const size_t MNP = (size_t)model->M * model->NP;
  HMM_CUDA(cudaMemsetAsync(stats->rec.p, 0, (size_t)model->M * rec_size(model->NP) * 8, st));
  if (model->table_family()) {
    stats->mv_rec.ensure(MNP * model->KS * 8);
    HMM_CUDA(cudaMemsetAsync(stats->mv_rec.p, 0, MNP * model->KS * 8, st));
  }
  if (model->any_support) {
    stats->ext_mm.ensure(MNP * 2 * 4);
    ext_support_init_kernel<<<(unsigned)((MNP + 127) / 128), 128, 0, st>>>(stats->ext_mm.as<int>(), (int)MNP);
    HMM_CUDA(cudaGetLastError());
  }
  stats->valid = true;
  stats->gamma_T = 0;
}

void prepare_mstep(hmm_model model, hmm_stats stats, const hmm_batch* b, hmm_plan plan) {
  if (!(model->any_negbin || model->any_weibull) || !b || (!plan && b->n_seq > 0)) return;
  const int RS = model->NP * 3;
  stats->dps.ensure((size_t)model->M * model->NP * sizeof(DPState));
  stats->dp_part.ensure((size_t)std::max<int64_t>(b->n_seq, 1) * RS * 4);
  stats->dp_chunk.ensure((size_t)std::max(plan ? plan->n_chunks : 0, 1) * RS * 8);
  stats->dp_rec.ensure((size_t)model->M * RS * 8);
  if (model->any_negbin) {
    stats->nb_hist.ensure((size_t)model->M * model->NP * NB_YMAX * 8);
    stats->nb_tail.ensure((size_t)std::max<int64_t>(b->n_seq, 1));
    HMM_CUDA(ensure_max_dyn_smem(reinterpret_cast<const void*>(nb_hist_kernel),
                                 (size_t)model->NP * NB_YMAX * 8));
  }
  stats->dp_count.ensure(64 * sizeof(int));
}

void run_mstep(hmm_ctx ctx, hmm_model model, hmm_stats stats, const MStepOpts& o_in, const hmm_batch* b,
               hmm_plan plan, cudaStream_t st) {
  MStepOpts o = o_in;
  o.hard = stats->hard ? 1 : 0;   // statistics of Viterbi paths: transition counts
  if (model->table_family()) HMM_REQUIRE(stats->mv_rec.p != nullptr, "table-family statistics were never computed");
  const bool dpass = model->any_negbin || model->any_weibull;
  if (dpass && model->NP > 32)
    throw Error{HMM_E_UNSUPPORTED, "Weibull / negative-binomial M-steps support padded N <= 32"};
  DPState* dps = nullptr;
  if (dpass) {
    HMM_REQUIRE(b != nullptr && (plan != nullptr || b->n_seq == 0),
                "Weibull / negative-binomial M-steps need the batch");
    HMM_REQUIRE(stats->gamma_T == b->total_T, "the statistics were not made from this batch");
    stats->dps.ensure((size_t)model->M * model->NP * sizeof(DPState));
    dps = stats->dps.as<DPState>();
  }
  {
    KTimer kt(ctx, HMM_KT_MSTEP, st);
    kt.kernels = 1 + 2 * (model->NP >= 16) + 2 * (int)model->any_discrete + 2 * (int)model->any_mv +
                 (int)model->any_ext +
                 2 * (int)model->any_indep;
    if (model->any_indep) {   // Sec. 4.5: every component's scalar update with the state's weights
      const int n = model->M * model->NP * model->D;
      indep_mstep_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->icomp.as<int>(), model->ishift.as<float>(),
                                                          model->theta.as<double>(), stats->mv_rec.as<double>(),
                                                          model->M, model->NP, model->N, model->P, model->D,
                                                          model->KS, o);
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_ext) {   // Sec. 4 / 4.2 closed forms and the chi-squared Newton; derived below
      const int n = model->M * model->NP;
      if (model->any_support) HMM_REQUIRE(stats->ext_mm.p != nullptr, "support statistics were never computed");
      ext_mstep_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->family.as<int>(), model->theta.as<double>(),
                                                        stats->mv_rec.as<double>(), stats->ext_mm.as<int>(),
                                                        model->M, model->NP, model->N, model->P, model->KS, o);
      HMM_CUDA(cudaGetLastError());
    }
    // from 16 states the transition rows and their float32 tables run as
    // their own kernels (one block per row, one thread per entry): one thread
    // per state would leave a single model's M-step on one SM, dominated by
    // the serial chain of its N float64 logarithms
    const bool rows_split = model->NP >= 16;
    mstep_kernel<<<model->M, model->NP, 0, st>>>(model->bufs(), stats->rec.as<double>(), o, dps, rows_split);
    HMM_CUDA(cudaGetLastError());
    if (rows_split) {
      mstep_rows_kernel<<<model->M * model->NP, 128, 0, st>>>(model->bufs(), stats->rec.as<double>(), o);
      HMM_CUDA(cudaGetLastError());
      const int64_t ne = (int64_t)model->M * model->NP * model->NP;
      derive_tables_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(model->bufs());
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_indep) {
      const int n = model->M * model->NP * model->D;
      indep_derive_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->icomp.as<int>(), model->theta.as<double>(),
                                                           model->M, model->NP, model->N, model->P, model->D,
                                                           model->icoef.as<float>(), model->ishift.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_discrete) {   // Sec. 4.1 "Discrete": weighted symbol frequencies
      const int n = model->M * model->NP;
      discrete_mstep_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->theta.as<double>(), stats->mv_rec.as<double>(),
                                                             model->M, model->NP, model->N, model->P, model->K,
                                                             o.collapse_eps);
      HMM_CUDA(cudaGetLastError());
      discrete_derive_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->theta.as<double>(), model->M, model->NP,
                                                              model->N, model->P, model->K, model->dtab.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_mv) {   // Sec. 4.5: means, (co)variances, then the new factors
      const int n = model->M * model->NP;
      mv_mstep_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->family.as<int>(), model->theta.as<double>(),
                                                       model->mvcoef.as<float>(), stats->mv_rec.as<double>(),
                                                       model->M, model->NP, model->N, model->P, model->D, model->KM,
                                                       model->KS, o.collapse_eps, o.tikhonov_eps);
      HMM_CUDA(cudaGetLastError());
      mv_derive_kernel<<<(n + 127) / 128, 128, 0, st>>>(model->family.as<int>(), model->theta.as<double>(),
                                                        model->M, model->NP, model->N, model->P, model->D, model->KM,
                                                        model->mvcoef.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
  }
  // an empty shard runs the passes only to take part in the exchange
  if (!dpass || (b->n_seq == 0 && !stats->reduce_fn)) return;
  // Newton steps that re-read the data: a fixed number of passes
  // (converged states skip their work), then the Weibull scale pass
  const int NP = model->NP, RS = NP * 3;
  const int64_t S = b->n_seq;
  stats->dp_part.ensure((size_t)std::max<int64_t>(S, 1) * RS * 4);
  stats->dp_chunk.ensure((size_t)std::max(plan ? plan->n_chunks : 0, 1) * RS * 8);
  stats->dp_rec.ensure((size_t)model->M * RS * 8);
  const int passes = std::min(o.newton_maxit, 24);   // + one final pass
  // a warp per sequence, grid-stride: passes after convergence exit in few blocks
  const unsigned blocks = (unsigned)std::min<int64_t>((S * 32 + 255) / 256, (int64_t)ctx->n_sm * 8);
  const int nthr = model->M * NP;
  KTimer kt(ctx, HMM_KT_MSTEP, st);
  kt.kernels = 2 + (int)model->any_negbin +
               (passes + 1) * ((int)model->any_negbin + (S > 0 ? 3 + (plan->n_chunks > 0) : 1));
  prepare_mstep(model, stats, b, plan);
  if (model->any_negbin && S > 0) {   // weighted histograms of the small counts, once per M-step
    HMM_CUDA(cudaMemsetAsync(stats->nb_hist.p, 0, (size_t)model->M * NP * NB_YMAX * 8, st));
    HMM_CUDA(cudaMemsetAsync(stats->nb_tail.p, 0, (size_t)S, st));
    if (plan->n_chunks > 0) {
      // row splits of about 4096 rows per chunk (at most 64)
      const int split = (int)std::min<int64_t>(64, std::max<int64_t>(1, (plan->max_chunk_rows + 4095) / 4096));
      nb_hist_kernel<<<dim3((unsigned)plan->n_chunks, (unsigned)split), 256, (size_t)NP * NB_YMAX * 8, st>>>(
          model->bufs(), b->values, stats->gamma.as<float>(), b->offsets, b->model_id,
          plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(), plan->chunk_hi.as<int32_t>(),
          plan->chunk_row0.as<int64_t>(), split, stats->nb_hist.as<unsigned long long>(), stats->nb_tail.as<uint8_t>());
      HMM_CUDA(cudaGetLastError());
    }
    kt.kernels += 3;
  }
  // active-state counters, one per pass (the update of pass p fills p + 1);
  // passes with no active state return at once
  int* cnt = stats->dp_count.as<int>();
  HMM_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(passes + 2) * sizeof(int), st));
  dp_count_kernel<<<(nthr + 127) / 128, 128, 0, st>>>(dps, nthr, cnt);
  HMM_CUDA(cudaGetLastError());
  for (int it = 0; it <= passes; ++it) {
    if (S > 0) {
      dp_sums_kernel<<<blocks, 256, 0, st>>>(model->bufs(), b->values, stats->gamma.as<float>(), b->offsets,
                                             b->model_id, (int)S, dps, stats->nb_tail.as<uint8_t>(), cnt + it,
                                             stats->dp_part.as<float>());
      HMM_CUDA(cudaGetLastError());
      if (plan->n_chunks > 0) {
        reduce_records_l1<<<plan->n_chunks, 128, 0, st>>>(stats->dp_part.as<float>(), RS,
                                                        plan->seq_by_model.as<int32_t>(),
                                                        plan->chunk_lo.as<int32_t>(), plan->chunk_hi.as<int32_t>(),
                                                        stats->dp_chunk.as<double>(), cnt + it);
        HMM_CUDA(cudaGetLastError());
      }
      reduce_chunks_l2<<<l2_grid(model->M, RS, 128), 128, 0, st>>>(stats->dp_chunk.as<double>(),
                                                                   plan->model_chunk_ptr.as<int32_t>(),
                                                 RS, stats->dp_rec.as<double>(), cnt + it);
      HMM_CUDA(cudaGetLastError());
      if (model->any_negbin) {   // the histogram rows of the negative-binomial sums
        const int nw = model->M * NP;
        nb_histdot_kernel<<<(unsigned)((nw * 32 + 255) / 256), 256, 0, st>>>(
            model->bufs(), dps, cnt + it, stats->nb_hist.as<unsigned long long>(), stats->dp_rec.as<double>());
        HMM_CUDA(cudaGetLastError());
      }
    } else {
      HMM_CUDA(cudaMemsetAsync(stats->dp_rec.p, 0, (size_t)model->M * RS * 8, st));
    }
    // this pass's sums over all processes' data before the update reads them
    call_reduce(stats, stats->dp_rec.p, (int64_t)model->M * RS, HMM_REDUCE_SUM_F64, st);
    dp_update_kernel<<<(nthr + 127) / 128, 128, 0, st>>>(model->bufs(), stats->dp_rec.as<double>(), dps, o,
                                                         it == passes ? 1 : 0, cnt + it, cnt + it + 1);
    HMM_CUDA(cudaGetLastError());
  }
  dp_finish_kernel<<<(nthr + 127) / 128, 128, 0, st>>>(model->bufs());
  HMM_CUDA(cudaGetLastError());
  if (model->any_negbin) {   // the count tables of the new r, one warp per state
    nb_table_kernel<<<(unsigned)((nthr * 32 + 255) / 256), 256, 0, st>>>(model->bufs());
    HMM_CUDA(cudaGetLastError());
  }
}

}  // namespace

const double* hmm::fit_async(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, hmm_stats stats,
                             const hmm_mstep_opts* opts, int iters, cudaStream_t st) {
  const MStepOpts mo = to_opts(opts);
  const int M = model->M, RS = rec_size(model->NP);
  ctx->trace.ensure((size_t)std::max(iters, 1) * M * 8 + 64);
  int* it_dev = reinterpret_cast<int*>(ctx->trace.as<char>() + (size_t)std::max(iters, 1) * M * 8);
  HMM_CUDA(cudaMemsetAsync(it_dev, 0, sizeof(int), st));
  prepare_mstep(model, stats, b, plan);
  for (int k = 0; k < iters; ++k) {
    run_estep(ctx, model, b, plan, nullptr, nullptr, nullptr, true, stats, st);
    trace_gather_kernel<<<(M + 255) / 256, 256, 0, st>>>(stats->rec.as<double>(), RS, M, ctx->trace.as<double>(),
                                                        it_dev);
    HMM_CUDA(cudaGetLastError());
    run_mstep(ctx, model, stats, mo, b, plan, st);
    bump_kernel<<<1, 1, 0, st>>>(it_dev);
    HMM_CUDA(cudaGetLastError());
  }
  return ctx->trace.as<double>();
}

void hmm::estep_async(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, hmm_stats stats,
                      double* d_loglik, cudaStream_t st) {
  run_estep(ctx, model, b, plan, nullptr, nullptr, d_loglik, true, stats, st);
}

// ================================================================ C ABI
extern "C" {

const char* hmm_status_string(hmm_status s) {
  switch (s) {
    case HMM_OK: return "ok";
    case HMM_E_ARG: return "invalid argument";
    case HMM_E_NOMEM: return "out of memory";
    case HMM_E_CUDA: return "CUDA error";
    case HMM_E_NUMERIC: return "non-finite result";
    case HMM_E_TIMEOUT: return "device wait timed out";
    case HMM_E_BUSY: return "queue full";
    case HMM_E_NOTREADY: return "not ready";
    case HMM_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* hmm_last_error(void) { return g_last_error.c_str(); }
const char* hmm_version(void) { return "hmmgpu 0.1 (sm_103a)"; }

int32_t hmm_family_param_count(int32_t family, int32_t dim) {
  if (family < 0 || family > HMM_PARETO) return -1;
  if (family >= HMM_DIAG_GAUSS && dim < 1) return -1;
  if (family == HMM_DISCRETE && (dim < 1 || dim > 1024)) return -1;
  return param_count(family, dim);
}

hmm_status hmm_information_criteria(int32_t family, int32_t n_states, int32_t dim, double loglik, int64_t n_obs,
                                    double* h_out) {
  return guarded([&] {
    HMM_REQUIRE(h_out != nullptr, "NULL argument");
    HMM_REQUIRE(n_states >= 1 && n_obs >= 1, "n_states and n_obs must be >= 1");
    const int pc = hmm_family_param_count(family, dim);
    HMM_REQUIRE(pc >= 0, "unknown family or dimension");
    int64_t e = pc;                                          // free emission parameters per state
    if (family == HMM_DISCRETE) e = dim - 1;                 // the K probabilities sum to 1
    if (family == HMM_FULL_GAUSS) e = dim + (int64_t)dim * (dim + 1) / 2;   // symmetric covariance
    const double N = n_states, n = (double)n_obs;
    const double k = (N - 1.0) + N * (N - 1.0) + N * (double)e;
    const double aic = 2.0 * k - 2.0 * loglik;
    h_out[0] = k;
    h_out[1] = aic;
    h_out[2] = k * std::log(n) - 2.0 * loglik;
    h_out[3] = (n - k - 1.0 > 0.0) ? aic + 2.0 * k * (k + 1.0) / (n - k - 1.0) : INFINITY;
  });
}

int64_t hmm_param_blob_size(int32_t n_models, int32_t n_states, int32_t dim, const int32_t* h_family) {
  if (n_models <= 0 || n_states <= 0 || !h_family) return -1;
  int64_t tot = 0;
  for (int m = 0; m < n_models; ++m) {
    const int pc = hmm_family_param_count(h_family[m], dim);
    if (pc < 0) return -1;
    tot += n_states + (int64_t)n_states * n_states + (int64_t)n_states * pc;
  }
  return tot;
}

hmm_status hmm_ctx_create(int device, size_t workspace_bytes, hmm_ctx* out) {
  return guarded([&] {
    HMM_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    HMM_CUDA(cudaGetDeviceCount(&ndev));
    HMM_REQUIRE(device >= 0 && device < ndev, "no such CUDA device");
    HMM_CUDA(cudaSetDevice(device));
    auto* c = new hmm_ctx_s();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->counters, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->counters, 0, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->work_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      if (c->status) cudaFree(c->status);
      if (c->counters) cudaFree(c->counters);
      delete c;
      throw Error{HMM_E_CUDA, std::string("context setup: ") + cudaGetErrorString(e)};
    }
    if (workspace_bytes) c->scratch.ensure(workspace_bytes);
    *out = c;
  });
}

hmm_status hmm_ctx_destroy(hmm_ctx ctx) {
  return guarded([&] {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    ctx->scratch.release();
    ctx->partials.release();
    ctx->chunk_rec.release();
    ctx->loglik.release();
    ctx->psi.release();
    ctx->gamma.release();
    ctx->dp_part.release();
    ctx->trace.release();
    cudaFree(ctx->status);
    cudaFree(ctx->counters);
    if (ctx->work_stream) cudaStreamDestroy(ctx->work_stream);
    for (auto& r : ctx->pending) {
      cudaEventDestroy(r.e0);
      cudaEventDestroy(r.e1);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    ctx->plain_beta.release();
    ctx->tune_out.release();
    ctx->mvlogb.release();
    ctx->lg_bv.release();
    ctx->lg_logAT.release();
    ctx->lg_off.release();
    ctx->lg_rz.release();
    ctx->lg_xi.release();
    ctx->xi_xt.release();
    ctx->xi_yt.release();
    ctx->vt_path.release();
    ctx->vt_count.release();
    for (auto* bb : {&ctx->km_u, &ctx->km_d2, &ctx->km_part, &ctx->km_flags}) bb->release();
    for (auto* bb : {&ctx->tp_Q, &ctx->tp_qexp, &ctx->tp_bvec, &ctx->tp_boff}) bb->release();
    delete ctx;
  });
}

hmm_status hmm_ctx_status(hmm_ctx ctx, void* stream) {
  int v = 0;
  hmm_status st = guarded([&] {
    HMM_REQUIRE(ctx != nullptr, "ctx is NULL");
    HMM_CUDA(cudaStreamSynchronize(S(stream)));
    HMM_CUDA(cudaMemcpy(&v, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    HMM_CUDA(cudaMemset(ctx->status, 0, sizeof(int)));
  });
  if (st != HMM_OK) return st;
  if (v & ST_TIMEOUT) return HMM_E_TIMEOUT;
  if (v & ST_NUMERIC) return HMM_E_NUMERIC;
  if (v & ST_ARG) return HMM_E_ARG;
  return HMM_OK;
}

hmm_status hmm_ctx_set_option(hmm_ctx ctx, int32_t key, int64_t value) {
  return guarded([&] {
    HMM_REQUIRE(ctx != nullptr, "ctx is NULL");
    switch (key) {
      case HMM_OPT_PROFILE: ctx->profile = value != 0; break;
      case HMM_OPT_ESTEP_LANES: ctx->estep_lanes = (int)value; break;
      case HMM_OPT_VITERBI_LANES: ctx->viterbi_lanes = (int)value; break;
      case HMM_OPT_PLAIN_ESTEP: ctx->plain_estep = value != 0; break;
      case HMM_OPT_TENSOR_RECURRENCE: ctx->tensor_rec = value == 2 ? 2 : (value != 0 ? 1 : 0); break;
      case HMM_OPT_TIME_PARALLEL: ctx->time_parallel = (int)value; break;
      default: throw Error{HMM_E_ARG, "unknown option"};
    }
  });
}

hmm_status hmm_ctx_profile_read(hmm_ctx ctx, double* h_ms, int64_t* h_launches, int32_t n_slots,
                                int32_t reset) {
  return guarded([&] {
    HMM_REQUIRE(ctx != nullptr, "ctx is NULL");
    for (auto& r : ctx->pending) {
      HMM_CUDA(cudaEventSynchronize(r.e1));
      float ms = 0.f;
      HMM_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
      if (r.slot >= 0 && r.slot < HMM_KT_SLOTS) {
        ctx->kt_ms[r.slot] += ms;
        ctx->kt_n[r.slot] += r.kernels;
      }
      ctx->event_pool.push_back(r.e0);
      ctx->event_pool.push_back(r.e1);
    }
    ctx->pending.clear();
    for (int i = 0; i < n_slots && i < HMM_KT_SLOTS; ++i) {
      if (h_ms) h_ms[i] = ctx->kt_ms[i];
      if (h_launches) h_launches[i] = ctx->kt_n[i];
    }
    if (reset)
      for (int i = 0; i < HMM_KT_SLOTS; ++i) {
        ctx->kt_ms[i] = 0.0;
        ctx->kt_n[i] = 0;
      }
  });
}

namespace {
// Model creation of hmm_model_create (h_comp == NULL) and
// hmm_model_create_indep (h_family all HMM_INDEP, h_comp [n_models][dim]).
void create_model(hmm_ctx ctx, int32_t n_models, int32_t n_states, int32_t dim, const int32_t* h_family,
                  const int32_t* h_comp, hmm_model* out) {
  {
    HMM_REQUIRE(ctx && out && h_family, "NULL argument");
    *out = nullptr;
    HMM_REQUIRE(n_models >= 1 && n_states >= 1 && n_states <= 1024 && dim >= 1, "bad model sizes");
    auto* m = new hmm_model_s();
    try {
      m->ctx = ctx;
      m->M = n_models;
      m->N = n_states;
      m->NP = padded_states(n_states);
      m->D = dim;
      m->dim_arg = dim;
      m->h_family.assign(h_family, h_family + n_models);
      int P = 1;
      if (h_comp) {   // independent components (Sec. 4.5)
        HMM_REQUIRE(dim <= INDEP_MAX_D, "independent components support dim <= 32");
        m->any_indep = true;
        m->h_icomp.assign(h_comp, h_comp + (size_t)n_models * dim);
        m->KS = 1;
        for (int i = 0; i < n_models; ++i) {
          int pc = 0, ks = 1;
          for (int d = 0; d < dim; ++d) {
            const int f = h_comp[(size_t)i * dim + d];
            if (!indep_component_ok(f))
              throw Error{HMM_E_UNSUPPORTED, "component family " + std::to_string(f) +
                                                 " is not supported in independent components"};
            pc += indep_param_count(f);
            ks += indep_stat_count(f);
          }
          P = std::max(P, pc);
          m->KS = std::max(m->KS, ks);
        }
      }
      for (int i = 0; i < n_models; ++i) {
        const int f = h_family[i];
        HMM_REQUIRE((h_comp != nullptr) == (f == HMM_INDEP), "HMM_INDEP models are made by hmm_model_create_indep");
        if (f == HMM_INDEP) continue;
        HMM_REQUIRE(f >= 0 && f <= HMM_PARETO, "unknown family");
        const bool mv = f == HMM_DIAG_GAUSS || f == HMM_FULL_GAUSS;
        HMM_REQUIRE(mv || f == HMM_DISCRETE || dim == 1, "scalar families need dim == 1");
        m->any_discrete |= f == HMM_DISCRETE;
        m->any_negbin |= f == HMM_NEGBIN;
        m->any_weibull |= f == HMM_WEIBULL;
        m->any_mv |= mv;
        m->any_ext |= is_ext_family(f);
        m->any_support |= ext_has_support_stats(f);
        P = std::max(P, param_count(f, dim));
      }
      for (int i = 0; i < n_models; ++i) {
        HMM_REQUIRE(!m->any_mv || h_family[i] == HMM_DIAG_GAUSS || h_family[i] == HMM_FULL_GAUSS,
                    "multivariate and scalar families cannot share a model set");
        HMM_REQUIRE(!m->any_discrete || h_family[i] == HMM_DISCRETE,
                    "the discrete family cannot share a model set with others");
        HMM_REQUIRE(!m->any_ext || is_ext_family(h_family[i]),
                    "log-normal .. Pareto share a model set only with each other");
      }
      if (m->any_ext)
        for (int i = 0; i < n_models; ++i) m->KS = std::max(m->KS, ext_stat_count(h_family[i]));
      if (m->any_discrete) {
        HMM_REQUIRE(dim >= 1 && dim <= 1024, "the discrete family needs 1 <= dim (symbols) <= 1024");
        m->K = dim;
        m->KS = dim;
        m->D = 1;                  // observations: one symbol index per step
      }
      m->P = P;
      const size_t M = n_models, NP = m->NP;
      m->family.ensure(M * 4);
      m->pi.ensure(M * NP * 8);
      m->A.ensure(M * NP * NP * 8);
      m->theta.ensure(M * NP * P * 8);
      m->A32.ensure(M * NP * NP * 4);
      if (NP > 32) m->AT32.ensure(M * NP * NP * 4);
      m->logA2.ensure(M * NP * NP * 4);
      m->logAe.ensure(M * NP * NP * 4);
      m->pi32.ensure(M * NP * 4);
      m->logpi2.ensure(M * NP * 4);
      m->logpie.ensure(M * NP * 4);
      m->coef.ensure(M * NP * KC * 4);
      if (m->any_negbin) m->nbtab.ensure(M * NP * NB_YMAX * 4);
      if (m->any_discrete) m->dtab.ensure(M * NP * (size_t)m->K * 4);
      if (m->any_mv) {
        HMM_REQUIRE(dim <= 32, "multivariate families support dim <= 32");
        for (int i = 0; i < n_models; ++i)
          if (h_family[i] == HMM_DIAG_GAUSS || h_family[i] == HMM_FULL_GAUSS) {
            m->KM = std::max(m->KM, mv_coef_count(h_family[i], dim));
            m->KS = std::max(m->KS, mv_stat_count(h_family[i], dim));
          }
        m->mvcoef.ensure(M * NP * m->KM * 4);
        HMM_CUDA(cudaMemset(m->mvcoef.p, 0, M * NP * m->KM * 4));
      }
      if (m->any_indep) {
        m->icomp.ensure(M * dim * 4);
        m->icoef.ensure(M * NP * dim * KC * 4);
        m->ishift.ensure(M * NP * dim * 4);
        HMM_CUDA(cudaMemcpy(m->icomp.p, h_comp, M * dim * 4, cudaMemcpyHostToDevice));
        HMM_CUDA(cudaMemset(m->icoef.p, 0, M * NP * dim * KC * 4));
        HMM_CUDA(cudaMemset(m->ishift.p, 0, M * NP * dim * 4));
      }
      m->lfact2.ensure(LF_YMAX * 4);
      HMM_CUDA(cudaMemcpy(m->family.p, h_family, M * 4, cudaMemcpyHostToDevice));
      HMM_CUDA(cudaMemset(m->pi.p, 0, M * NP * 8));
      HMM_CUDA(cudaMemset(m->A.p, 0, M * NP * NP * 8));
      HMM_CUDA(cudaMemset(m->theta.p, 0, M * NP * P * 8));
      HMM_CUDA(cudaMemset(m->coef.p, 0, M * NP * KC * 4));
      lfact_kernel<<<(LF_YMAX + 255) / 256, 256>>>(m->lfact2.as<float>());
      HMM_CUDA(cudaGetLastError());
      HMM_CUDA(cudaStreamSynchronize(0));
    } catch (...) {
      for (auto* b : {&m->family, &m->pi, &m->A, &m->theta, &m->A32, &m->AT32, &m->logA2, &m->logAe, &m->pi32,
                      &m->logpi2, &m->logpie, &m->coef, &m->nbtab, &m->lfact2, &m->mvcoef, &m->dtab, &m->icomp,
                      &m->icoef, &m->ishift})
        b->release();
      delete m;
      throw;
    }
    *out = m;
  }
}
}  // namespace

hmm_status hmm_model_create(hmm_ctx ctx, int32_t n_models, int32_t n_states, int32_t dim,
                            const int32_t* h_family, hmm_model* out) {
  return guarded([&] { create_model(ctx, n_models, n_states, dim, h_family, nullptr, out); });
}

hmm_status hmm_model_create_indep(hmm_ctx ctx, int32_t n_models, int32_t n_states, int32_t dim,
                                  const int32_t* h_comp, hmm_model* out) {
  return guarded([&] {
    HMM_REQUIRE(h_comp != nullptr && n_models >= 1 && n_models <= (1 << 24), "NULL argument or bad model count");
    std::vector<int32_t> fam((size_t)n_models, HMM_INDEP);
    create_model(ctx, n_models, n_states, dim, fam.data(), h_comp, out);
  });
}

int64_t hmm_model_blob_size(hmm_model model) { return model ? model_blob_size(model) : -1; }

hmm_status hmm_model_destroy(hmm_model m) {
  return guarded([&] {
    if (!m) return;
    for (auto* b : {&m->family, &m->pi, &m->A, &m->theta, &m->A32, &m->AT32, &m->logA2, &m->logAe, &m->pi32,
                    &m->logpi2, &m->logpie, &m->coef, &m->nbtab, &m->lfact2, &m->mvcoef, &m->dtab, &m->icomp,
                    &m->icoef, &m->ishift})
      b->release();
    delete m;
  });
}

hmm_status hmm_model_set_params(hmm_model model, const double* h_blob, int64_t n_values) {
  return guarded([&] {
    HMM_REQUIRE(model && h_blob, "NULL argument");
    const int M = model->M, N = model->N, NP = model->NP, P = model->P, D = model->D;
    const int64_t need = model_blob_size(model);
    HMM_REQUIRE(n_values == need, "parameter blob has the wrong size");
    std::vector<double> pi((size_t)M * NP, 0.0), A((size_t)M * NP * NP, 0.0), th((size_t)M * NP * P, 0.0);
    const double* q = h_blob;
    for (int m = 0; m < M; ++m) {
      const int pc = model_param_count(model, m);
      double psum = 0.0;
      for (int j = 0; j < N; ++j) {
        HMM_REQUIRE(q[j] >= 0.0 && std::isfinite(q[j]), "pi must be finite and >= 0");
        pi[(size_t)m * NP + j] = q[j];
        psum += q[j];
      }
      HMM_REQUIRE(std::fabs(psum - 1.0) < 1e-6, "pi must sum to 1");
      q += N;
      for (int i = 0; i < N; ++i) {
        double rs = 0.0;
        for (int j = 0; j < N; ++j) {
          HMM_REQUIRE(q[j] >= 0.0 && std::isfinite(q[j]), "A must be finite and >= 0");
          A[((size_t)m * NP + i) * NP + j] = q[j];
          rs += q[j];
        }
        HMM_REQUIRE(std::fabs(rs - 1.0) < 1e-6, "rows of A must sum to 1");
        q += N;
      }
      for (int j = 0; j < N; ++j) {
        double psum = 0.0;
        for (int z = 0; z < pc; ++z) {
          HMM_REQUIRE(std::isfinite(q[z]), "parameters must be finite");
          th[((size_t)m * NP + j) * P + z] = q[z];
          psum += q[z];
          if (model->h_family[m] == HMM_DISCRETE) HMM_REQUIRE(q[z] >= 0.0, "symbol probabilities must be >= 0");
        }
        if (model->h_family[m] == HMM_DISCRETE)
          HMM_REQUIRE(std::fabs(psum - 1.0) < 1e-6, "symbol probabilities must sum to 1");
        if (model->h_family[m] == HMM_INDEP) {
          const double* qc = q;
          for (int d = 0; d < D; ++d) {
            const int f = model->h_icomp[(size_t)m * D + d];
            check_scalar_params(f, qc);
            qc += indep_param_count(f);
          }
        } else {
          check_scalar_params(model->h_family[m], q);
        }
        q += pc;
      }
    }
    HMM_CUDA(cudaMemcpy(model->pi.p, pi.data(), pi.size() * 8, cudaMemcpyHostToDevice));
    HMM_CUDA(cudaMemcpy(model->A.p, A.data(), A.size() * 8, cudaMemcpyHostToDevice));
    HMM_CUDA(cudaMemcpy(model->theta.p, th.data(), th.size() * 8, cudaMemcpyHostToDevice));
    const int n = M * NP;
    // from 16 states the transition tables run one thread per entry (as in
    // the M-step) instead of a float64 logarithm chain per state
    derive_kernel<<<(n + 127) / 128, 128>>>(model->bufs(), NP < 16);
    HMM_CUDA(cudaGetLastError());
    if (NP >= 16) {
      const int64_t ne = (int64_t)M * NP * NP;
      derive_tables_kernel<<<(unsigned)((ne + 255) / 256), 256>>>(model->bufs());
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_mv) {
      mv_derive_kernel<<<(n + 127) / 128, 128>>>(model->family.as<int>(), model->theta.as<double>(), M, NP, N, P, D,
                                                 model->KM, model->mvcoef.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_discrete) {
      discrete_derive_kernel<<<(n + 127) / 128, 128>>>(model->theta.as<double>(), M, NP, N, P, model->K,
                                                       model->dtab.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
    if (model->any_indep) {
      const int ni = n * D;
      indep_derive_kernel<<<(ni + 127) / 128, 128>>>(model->icomp.as<int>(), model->theta.as<double>(), M, NP, N, P,
                                                     D, model->icoef.as<float>(), model->ishift.as<float>());
      HMM_CUDA(cudaGetLastError());
    }
    // the copies and derive kernels ran on the legacy default stream
    HMM_CUDA(cudaStreamSynchronize(0));
  });
}

hmm_status hmm_model_get_params(hmm_model model, double* h_blob, int64_t n_values) {
  return guarded([&] {
    HMM_REQUIRE(model && h_blob, "NULL argument");
    const int M = model->M, N = model->N, NP = model->NP, P = model->P;
    const int64_t need = model_blob_size(model);
    HMM_REQUIRE(n_values == need, "parameter blob has the wrong size");
    HMM_CUDA(cudaDeviceSynchronize());
    std::vector<double> pi((size_t)M * NP), A((size_t)M * NP * NP), th((size_t)M * NP * P);
    HMM_CUDA(cudaMemcpy(pi.data(), model->pi.p, pi.size() * 8, cudaMemcpyDeviceToHost));
    HMM_CUDA(cudaMemcpy(A.data(), model->A.p, A.size() * 8, cudaMemcpyDeviceToHost));
    HMM_CUDA(cudaMemcpy(th.data(), model->theta.p, th.size() * 8, cudaMemcpyDeviceToHost));
    double* q = h_blob;
    for (int m = 0; m < M; ++m) {
      const int pc = model_param_count(model, m);
      for (int j = 0; j < N; ++j) *q++ = pi[(size_t)m * NP + j];
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) *q++ = A[((size_t)m * NP + i) * NP + j];
      for (int j = 0; j < N; ++j)
        for (int z = 0; z < pc; ++z) *q++ = th[((size_t)m * NP + j) * P + z];
    }
  });
}

hmm_status hmm_plan_create(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, const int64_t* h_offsets,
                           const int32_t* h_model_id, hmm_plan* out) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && batch && out, "NULL argument");
    *out = nullptr;
    check_batch(model, batch);
    *out = make_plan(ctx, model, batch, h_offsets, h_model_id);
  });
}

hmm_status hmm_plan_destroy(hmm_plan plan) {
  return guarded([&] { destroy_plan(plan); });
}

hmm_status hmm_plan_autotune(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, double* h_ms, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && batch && batch->plan, "NULL argument (the batch needs a plan)");
    check_batch(model, batch);
    hmm_plan plan = batch->plan;
    HMM_REQUIRE(plan->n_seq == batch->n_seq && plan->total_T == batch->total_T, "plan does not match the batch");
    if (model->NP > 32 || batch->n_seq == 0) return;
    cudaStream_t st = S(stream);
    const int NP = model->NP;
    ctx->tune_out.ensure((size_t)std::max<int64_t>(batch->total_T, 1) * 4 + (size_t)batch->n_seq * 8 + 256);
    int32_t* path = ctx->tune_out.as<int32_t>();
    double* score = reinterpret_cast<double*>(ctx->tune_out.as<char>() +
                                              (((size_t)std::max<int64_t>(batch->total_T, 1) * 4 + 255) & ~size_t(255)));
    cudaEvent_t e0, e1;
    HMM_CUDA(cudaEventCreate(&e0));
    HMM_CUDA(cudaEventCreate(&e1));
    struct Ev {
      cudaEvent_t a, b;
      ~Ev() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
      }
    } ev{e0, e1};
    const int saved_e = ctx->estep_lanes, saved_v = ctx->viterbi_lanes, saved_p = ctx->plain_estep;
    ctx->plain_estep = 0;
    double best_e = 1e30, best_v = 1e30;
    int g_e = 0, g_v = 0;
    try {
      for (int G = 1; G <= 16; G *= 2) {
        if (estep_small_supported(NP, G)) {
          ctx->estep_lanes = G;
          float ms = 0.f;
          for (int rep = 0; rep < 2; ++rep) {
            HMM_CUDA(cudaEventRecord(e0, st));
            run_estep(ctx, model, batch, plan, nullptr, nullptr, nullptr, false, nullptr, st);
            HMM_CUDA(cudaEventRecord(e1, st));
            HMM_CUDA(cudaEventSynchronize(e1));
            HMM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          }
          if (ms < best_e) {
            best_e = ms;
            g_e = G;
          }
        }
        if (viterbi_small_supported(NP, G)) {
          ctx->viterbi_lanes = G;
          float ms = 0.f;
          for (int rep = 0; rep < 2; ++rep) {
            HMM_CUDA(cudaEventRecord(e0, st));
            hmm_status vs = hmm_viterbi(ctx, model, batch, nullptr, path, score, stream);
            if (vs != HMM_OK) throw Error{vs, hmm_last_error()};
            HMM_CUDA(cudaEventRecord(e1, st));
            HMM_CUDA(cudaEventSynchronize(e1));
            HMM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          }
          if (ms < best_v) {
            best_v = ms;
            g_v = G;
          }
        }
      }
    } catch (...) {
      ctx->estep_lanes = saved_e;
      ctx->viterbi_lanes = saved_v;
      ctx->plain_estep = saved_p;
      throw;
    }
    ctx->estep_lanes = saved_e;
    ctx->viterbi_lanes = saved_v;
    ctx->plain_estep = saved_p;
    plan->estep_G = g_e;
    plan->viterbi_G = g_v;
    if (h_ms) {
      h_ms[0] = best_e;
      h_ms[1] = best_v;
    }
  });
}

hmm_status hmm_emission_logpdf(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, float* d_logb,
                               void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && d_logb, "NULL argument");
    check_batch(model, batch);
    if (batch->n_seq == 0) return;
    PlanRef prr;
    get_plan(ctx, model, batch, S(stream), prr);
    const unsigned slabs = slabs_of(prr.p->max_T);
    if (model->any_indep) {
      KTimer kt(ctx, HMM_KT_EMISSION, S(stream));
      launch_indep_emission(model, batch, prr.p, d_logb, S(stream));
      if (prr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
      return;
    }
    if (model->any_discrete) {
      KTimer kt(ctx, HMM_KT_EMISSION, S(stream));
      discrete_emission_kernel<<<dim3((unsigned)batch->n_seq, slabs), 128, 0, S(stream)>>>(
          model->dtab.as<float>(), model->NP, model->N, model->K, batch->values, batch->offsets, batch->model_id,
          d_logb);
      HMM_CUDA(cudaGetLastError());
      if (prr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
      return;
    }
    if (model->any_mv) {
      if (prr.p->n_tiles > 0) {
        KTimer kt(ctx, HMM_KT_EMISSION, S(stream));
        launch_mv_emission(model, batch, prr.p, d_logb, S(stream));
      }
      if (prr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
      return;
    }
    KTimer kt(ctx, HMM_KT_EMISSION, S(stream));
    emission_kernel<<<dim3((unsigned)batch->n_seq, slabs), 128, 0, S(stream)>>>(model->view(), batch->values,
                                                                             batch->offsets, batch->model_id, d_logb);
    HMM_CUDA(cudaGetLastError());
  });
}

hmm_status hmm_forward_backward(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, const float* d_logb,
                                float* d_gamma, int32_t* d_post_path, double* d_loglik, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && d_loglik, "NULL argument");
    check_batch(model, batch);
    PlanRef pr;
    get_plan(ctx, model, batch, S(stream), pr);
    float* gamma = d_gamma;
    if (!gamma && d_post_path) {
      ctx->gamma.ensure(std::max<int64_t>(batch->total_T, 1) * model->N * 4);
      gamma = ctx->gamma.as<float>();
    }
    run_estep(ctx, model, batch, pr.p, d_logb, gamma, d_loglik, false, nullptr, S(stream));
    if (d_post_path && batch->total_T > 0) {
      const unsigned blocks = (unsigned)((batch->total_T + 255) / 256);
      post_path_kernel<<<blocks, 256, 0, S(stream)>>>(gamma, batch->total_T, model->N, d_post_path);
      HMM_CUDA(cudaGetLastError());
    }
    if (pr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
  });
}

namespace {
// Viterbi decode of a batch (the body of hmm_viterbi) with a plan.
void run_viterbi(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, hmm_plan plan, const float* d_logb,
                 int32_t* d_path, double* d_score, cudaStream_t st) {
  const int64_t Sn = batch->n_seq;
  if (Sn == 0) return;
  if (model->NP > 32) {
    if (!d_logb) d_logb = mv_table(ctx, model, batch, plan, st);
    ctx->psi.ensure(std::max<int64_t>(batch->total_T, 1) * model->NP * 4 + 64);
    ctx->lg_logAT.ensure((size_t)model->M * model->NP * model->NP * 4);
    LargeArgs a{};
    a.logb = d_logb;
    a.offsets = batch->offsets;
    a.model_id = batch->model_id;
    a.groups = plan->lg_groups.as<int32_t>();
    a.n_groups = plan->n_groups;
    a.group_fill = plan->lg_fill;
    a.status = ctx->status;
    a.mv = model->view();
    a.psi = ctx->psi.as<uint16_t>();
    a.drow = ctx->psi.as<float>();
    a.logAT = ctx->lg_logAT.as<float>();
    a.path = d_path;
    a.score = d_score;
    KTimer kt(ctx, HMM_KT_VITERBI, st);
    HMM_CUDA(launch_large_viterbi(model->NP, a, st));
    return;
  }
  if (model->table_family() && !d_logb) d_logb = mv_table(ctx, model, batch, plan, st);
  const int NP = model->NP;
  ctx->psi.ensure(std::max<int64_t>(batch->total_T, 1) * NP + 64);
  VitArgs a;
  a.y = batch->values;
  a.logb = d_logb;
  a.offsets = batch->offsets;
  a.model_id = batch->model_id;
  a.order = plan->order.as<int32_t>();
  a.n_seq = (int32_t)Sn;
  int G = plan->viterbi_G > 0 ? plan->viterbi_G : default_viterbi_G(NP, Sn, ctx->n_sm);
  if (ctx->viterbi_lanes && viterbi_small_supported(NP, ctx->viterbi_lanes)) G = ctx->viterbi_lanes;
  a.n_items = (int32_t)((Sn + viterbi_seqs_per_item(G) - 1) / viterbi_seqs_per_item(G));
  a.mv = model->view();
  a.psi = ctx->psi.as<uint8_t>();
  a.path = d_path;
  a.score = d_score;
  a.work_counter = ctx->counters + 1;
  a.status = ctx->status;
  if (plan->n_fam_seg > 0) {
    a.sched.n_seg = plan->n_fam_seg;
    a.sched.seg_seq = plan->fam_seg_seq.as<int32_t>();
    a.sched.seg_sm = plan->fam_seg_sm.as<int32_t>();
    a.work_counter = ctx->counters + 16;
  }
  HMM_CUDA(cudaMemsetAsync(a.work_counter, 0, sizeof(int) * std::max(a.sched.n_seg, 1), st));
  KTimer kt(ctx, HMM_KT_VITERBI, st);
  const int fam = d_logb ? FAM_TABLE : (plan->uniform_family >= 0 ? plan->uniform_family : FAM_ANY);
  HMM_CUDA(launch_viterbi_small(NP, G, a, fam, ctx->n_sm, st));
}

// One-hot occupancies of decoded paths: gamma[t][j] = 1[path_t = j].
__global__ void onehot_kernel(const int32_t* __restrict__ path, int64_t total_T, int N, float* __restrict__ gamma) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total_T * N) return;
  gamma[i] = path[i / N] == (int32_t)(i % N) ? 1.f : 0.f;
}

// Transition counts of the decoded paths per 64-sequence chunk, as float64
// blocks [n_chunks][NP][NP] (integer atomics: exact, order-independent).
__global__ void path_xi_kernel(const int32_t* __restrict__ path, const int64_t* __restrict__ offsets,
                               const int32_t* __restrict__ seq_by_model, const int32_t* __restrict__ chunk_lo,
                               const int32_t* __restrict__ chunk_hi, int NP, int* __restrict__ counts,
                               double* __restrict__ xi_chunk) {
  const int c = blockIdx.x;
  int* cnt = counts + (size_t)c * NP * NP;
  for (int z = threadIdx.x; z < NP * NP; z += blockDim.x) cnt[z] = 0;
  __syncthreads();
  for (int qs = chunk_lo[c]; qs < chunk_hi[c]; ++qs) {
    const int s = seq_by_model[qs];
    const int64_t b = offsets[s], e = offsets[s + 1];
    for (int64_t t = b + threadIdx.x; t + 1 < e; t += blockDim.x) {
      const int i = path[t], j = path[t + 1];
      if (i >= 0 && i < NP && j >= 0 && j < NP) atomicAdd(&cnt[i * NP + j], 1);
    }
  }
  __syncthreads();
  double* out = xi_chunk + (size_t)c * NP * NP;
  for (int z = threadIdx.x; z < NP * NP; z += blockDim.x) out[z] = (double)cnt[z];
}

// Statistics of the Viterbi paths into `stats` (hmm_estep_viterbi).
void run_estep_viterbi(hmm_ctx ctx, hmm_model model, const hmm_batch* b, hmm_plan plan, hmm_stats stats,
                       double* d_score, cudaStream_t st) {
  const int NP = model->NP, N = model->N;
  const int64_t S = b->n_seq, TT = std::max<int64_t>(b->total_T, 1);
  ctx->vt_path.ensure((size_t)TT * 4);
  if (!d_score) {
    ctx->loglik.ensure(std::max<int64_t>(S, 1) * 8);
    d_score = ctx->loglik.as<double>();
  }
  run_viterbi(ctx, model, b, plan, nullptr, ctx->vt_path.as<int32_t>(), d_score, st);
  stats->gamma.ensure((size_t)TT * N * 4);
  stats->gamma_T = b->total_T;
  ctx->partials.ensure((size_t)std::max<int64_t>(S, 1) * NP * NST * 4);
  const int nc = plan->n_chunks;
  ctx->lg_xi.ensure((size_t)std::max(nc, 1) * NP * NP * 8);
  ctx->vt_count.ensure((size_t)std::max(nc, 1) * NP * NP * 4);
  ctx->chunk_rec.ensure((size_t)std::max(nc, 1) * rec_size(NP) * 8);
  KTimer kt(ctx, HMM_KT_REDUCE, st);
  kt.kernels = 3;
  const int64_t n = b->total_T * N;
  if (n > 0) {
    onehot_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->vt_path.as<int32_t>(), b->total_T, N,
                                                              stats->gamma.as<float>());
    HMM_CUDA(cudaGetLastError());
    ++kt.kernels;
  }
  LargeArgs a{};
  a.offsets = b->offsets;
  a.model_id = b->model_id;
  a.mv = model->view();
  HMM_CUDA(launch_large_stats(a, b->values, stats->gamma.as<float>(), S, model->table_family(),
                              ctx->partials.as<float>(), st));
  if (nc > 0) {
    path_xi_kernel<<<nc, 256, 0, st>>>(ctx->vt_path.as<int32_t>(), b->offsets, plan->seq_by_model.as<int32_t>(),
                                       plan->chunk_lo.as<int32_t>(), plan->chunk_hi.as<int32_t>(), NP,
                                       ctx->vt_count.as<int>(), ctx->lg_xi.as<double>());
    HMM_CUDA(cudaGetLastError());
    HMM_CUDA(launch_large_reduce(ctx->partials.as<float>(), d_score, ctx->lg_xi.as<double>(),
                                 plan->seq_by_model.as<int32_t>(), plan->chunk_lo.as<int32_t>(),
                                 plan->chunk_hi.as<int32_t>(), nc, NP, ctx->chunk_rec.as<double>(), st));
  }
  reduce_chunks_l2<<<l2_grid(model->M, rec_size(NP), 256), 256, 0, st>>>(ctx->chunk_rec.as<double>(),
                                                                         plan->model_chunk_ptr.as<int32_t>(),
                                             rec_size(NP), stats->rec.as<double>());
  HMM_CUDA(cudaGetLastError());
  if (model->table_family()) kt.kernels += mv_statistics(ctx, model, b, plan, stats, st);
  stats->valid = true;
  stats->hard = true;
}
}  // namespace

hmm_status hmm_viterbi(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, const float* d_logb,
                       int32_t* d_path, double* d_score, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && d_path && d_score, "NULL argument");
    check_batch(model, batch);
    PlanRef pr;
    get_plan(ctx, model, batch, S(stream), pr);
    run_viterbi(ctx, model, batch, pr.p, d_logb, d_path, d_score, S(stream));
    if (pr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
  });
}

hmm_status hmm_estep_viterbi(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, hmm_stats stats,
                             double* d_score, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && stats, "NULL argument");
    HMM_REQUIRE(stats->model == model, "stats belong to another model");
    check_batch(model, batch);
    if (batch->n_seq == 0) {
      zero_stats(model, stats, S(stream));
      stats->hard = true;
    } else {
      PlanRef pr;
      get_plan(ctx, model, batch, S(stream), pr);
      run_estep_viterbi(ctx, model, batch, pr.p, stats, d_score, S(stream));
      if (pr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
    }
    for (int i = 0; i < 3; ++i) {
      void* p = nullptr;
      int64_t n = 0;
      int op = 0;
      record_view(stats, i, &p, &n, &op);
      call_reduce(stats, p, n, op, S(stream));
    }
  });
}

hmm_status hmm_stats_create(hmm_ctx ctx, hmm_model model, hmm_stats* out) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && out, "NULL argument");
    auto* s = new hmm_stats_s();
    s->model = model;
    try {
      s->rec.ensure((size_t)model->M * rec_size(model->NP) * 8);
      HMM_CUDA(cudaMemset(s->rec.p, 0, (size_t)model->M * rec_size(model->NP) * 8));
    } catch (...) {
      s->rec.release();
      delete s;
      throw;
    }
    *out = s;
  });
}

hmm_status hmm_stats_destroy(hmm_stats stats) {
  return guarded([&] {
    if (!stats) return;
    for (auto* bb : {&stats->rec, &stats->gamma, &stats->dps, &stats->dp_part, &stats->dp_chunk, &stats->dp_rec,
                     &stats->dp_count, &stats->mv_part, &stats->mv_split, &stats->mv_chunk, &stats->mv_rec,
                     &stats->ext_mm, &stats->nb_hist, &stats->nb_tail})
      bb->release();
    delete stats;
  });
}

// inverse of the device's ordered float keys (support min / max)
static double ext_unkey_host(int k) {
  const uint32_t u = (uint32_t)(k >= 0 ? k : k ^ 0x7fffffff);
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

static int canon_fam_count(int fam, int D) {
  switch (fam) {
    case HMM_DISCRETE: return D;   // D: the model's dim (number of symbols)
    case HMM_GAUSS: return 3;
    case HMM_POISSON: return 2;
    case HMM_GAMMA: return 4;
    case HMM_BETA: return 5;
    case HMM_WEIBULL: return 3;
    case HMM_NEGBIN: return 3;
    case HMM_STUDENT_T: return 5;
    case HMM_VONMISES: return 3;
    case HMM_DIAG_GAUSS: return 1 + 2 * D;
    case HMM_FULL_GAUSS: return 1 + D + D * D;
    case HMM_LOGNORMAL: return 3;
    case HMM_EXPONENTIAL: return 2;
    case HMM_RAYLEIGH: return 2;
    case HMM_UNIFORM: return 3;
    case HMM_CHISQ: return 2;
    case HMM_PARETO: return 3;
  }
  return 0;
}

// Canonical statistics per state of model i (hmm_stats_get).
static int canon_count(hmm_model md, int i) {
  if (md->h_family[i] != HMM_INDEP) return canon_fam_count(md->h_family[i], md->dim_arg);
  int n = 1;
  for (int d = 0; d < md->D; ++d) n += indep_stat_count(md->h_icomp[(size_t)i * md->D + d]);
  return n;
}

int64_t hmm_stats_size(hmm_stats stats) {
  if (!stats) return -1;
  const hmm_model m = stats->model;
  int64_t tot = 0;
  for (int i = 0; i < m->M; ++i) tot += 2 + m->N + (int64_t)m->N * m->N + (int64_t)m->N * canon_count(m, i);
  return tot;
}

hmm_status hmm_stats_get(hmm_stats stats, double* h_out, int64_t n_values) {
  return guarded([&] {
    HMM_REQUIRE(stats && h_out, "NULL argument");
    HMM_REQUIRE(n_values == hmm_stats_size(stats), "output has the wrong size");
    HMM_REQUIRE(stats->valid, "statistics were never computed");
    const hmm_model md = stats->model;
    const int M = md->M, N = md->N, NP = md->NP, RS = rec_size(NP);
    HMM_CUDA(cudaDeviceSynchronize());
    std::vector<double> rec((size_t)M * RS), A((size_t)M * NP * NP);
    std::vector<float> coef((size_t)M * NP * KC);
    HMM_CUDA(cudaMemcpy(rec.data(), stats->rec.p, rec.size() * 8, cudaMemcpyDeviceToHost));
    HMM_CUDA(cudaMemcpy(A.data(), md->A.p, A.size() * 8, cudaMemcpyDeviceToHost));
    HMM_CUDA(cudaMemcpy(coef.data(), md->coef.p, coef.size() * 4, cudaMemcpyDeviceToHost));
    const int D = md->D, KM = md->KM, KS = md->KS;
    std::vector<double> mrec;
    std::vector<float> mvc;
    std::vector<int> emm;
    if (md->table_family()) {
      HMM_REQUIRE(stats->mv_rec.p != nullptr, "table-family statistics were never computed");
      mrec.resize((size_t)M * NP * KS);
      HMM_CUDA(cudaMemcpy(mrec.data(), stats->mv_rec.p, mrec.size() * 8, cudaMemcpyDeviceToHost));
      if (md->any_support) {
        HMM_REQUIRE(stats->ext_mm.p != nullptr, "support statistics were never computed");
        emm.resize((size_t)M * NP * 2);
        HMM_CUDA(cudaMemcpy(emm.data(), stats->ext_mm.p, emm.size() * 4, cudaMemcpyDeviceToHost));
      }
      if (md->any_mv) {
        mvc.resize((size_t)M * NP * KM);
        HMM_CUDA(cudaMemcpy(mvc.data(), md->mvcoef.p, mvc.size() * 4, cudaMemcpyDeviceToHost));
      }
    }
    std::vector<float> ish;
    if (md->any_indep) {
      ish.resize((size_t)M * NP * D);
      HMM_CUDA(cudaMemcpy(ish.data(), md->ishift.p, ish.size() * 4, cudaMemcpyDeviceToHost));
    }
    double* q = h_out;
    for (int m = 0; m < M; ++m) {
      const double* R = rec.data() + (size_t)m * RS;
      *q++ = R[0];
      *q++ = R[1];
      for (int j = 0; j < N; ++j) *q++ = R[rec_g1(NP) + j];
      for (int i = 0; i < N; ++i)   // expected transitions a_ij X_ij (counts after hmm_estep_viterbi)
        for (int j = 0; j < N; ++j)
          *q++ = (stats->hard ? 1.0 : A[((size_t)m * NP + i) * NP + j]) * R[rec_xi(NP) + i * NP + j];
      const int fam = md->h_family[m];
      for (int j = 0; j < N; ++j) {
        const double* St = R + rec_st(NP) + j * (NST - 1);
        const double c0 = coef[((size_t)m * NP + j) * KC];
        const double W = St[0];
        if (fam == HMM_INDEP) {   // W, then each component's sums, shifts undone
          const double* Rm = mrec.data() + ((size_t)m * NP + j) * KS;
          q[0] = Rm[0];
          int o = 1;
          for (int d = 0; d < D; ++d) {
            const int f = md->h_icomp[(size_t)m * D + d];
            const double c = ish[((size_t)m * NP + j) * D + d];
            const double* Sd = Rm + o;
            double* qd = q + o;
            const int n = indep_stat_count(f);
            for (int z = 0; z < n; ++z) qd[z] = Sd[z];
            if (f == HMM_GAUSS || f == HMM_LOGNORMAL) {
              qd[0] = Sd[0] + c * Rm[0];
              qd[1] = Sd[1] + 2.0 * c * Sd[0] + c * c * Rm[0];
            } else if (f == HMM_STUDENT_T) {
              qd[1] = Sd[1] + c * Sd[0];
              qd[2] = Sd[2] + 2.0 * c * Sd[1] + c * c * Sd[0];
            }
            o += n;
          }
          q += canon_count(md, m);
          continue;
        }
        switch (fam) {
          case HMM_GAUSS:   // shifted by c0: sum w d, sum w d^2 -> raw moments
            q[0] = W;
            q[1] = St[1] + c0 * W;
            q[2] = St[2] + 2 * c0 * St[1] + c0 * c0 * W;
            break;
          case HMM_POISSON:
            q[0] = W;
            q[1] = St[1];
            break;
          case HMM_GAMMA:
            q[0] = W;
            q[1] = St[1];
            q[2] = St[2] * kLn2;
            q[3] = St[3];
            break;
          case HMM_BETA:
            q[0] = W;
            q[1] = St[1];
            q[2] = St[2];
            q[3] = St[3] * kLn2;
            q[4] = St[4] * kLn2;
            break;
          case HMM_WEIBULL:
            q[0] = W;
            q[1] = St[1] * kLn2;
            q[2] = St[2] * kLn2 * kLn2;
            break;
          case HMM_NEGBIN:
            q[0] = W;
            q[1] = St[1];
            q[2] = St[2];
            break;
          case HMM_STUDENT_T:
            q[0] = W;
            q[1] = St[1];
            q[2] = St[2] + c0 * St[1];
            q[3] = St[3] + 2 * c0 * St[2] + c0 * c0 * St[1];
            q[4] = St[4];
            break;
          case HMM_VONMISES:
            q[0] = W;
            q[1] = St[1];
            q[2] = St[2];
            break;
          case HMM_DISCRETE: {   // weighted symbol counts
            const double* Rm = mrec.data() + ((size_t)m * NP + j) * KS;
            for (int k = 0; k < md->K; ++k) q[k] = Rm[k];
            break;
          }
          case HMM_LOGNORMAL:
          case HMM_EXPONENTIAL:
          case HMM_RAYLEIGH:
          case HMM_CHISQ:
          case HMM_UNIFORM:
          case HMM_PARETO: {   // feature sums, then the support min / max
            const double* Rm = mrec.data() + ((size_t)m * NP + j) * KS;
            const int nf = ext_stat_count(fam);
            for (int k = 0; k < nf; ++k) q[k] = Rm[k];
            if (fam == HMM_UNIFORM || fam == HMM_PARETO) {
              const int* g = emm.data() + ((size_t)m * NP + j) * 2;
              q[nf] = ext_unkey_host(g[0]);
              if (fam == HMM_UNIFORM) q[nf + 1] = ext_unkey_host(~g[1]);
            }
            break;
          }
          case HMM_DIAG_GAUSS:
          case HMM_FULL_GAUSS: {
            // raw moments W, sum g y_d, then sum g y_d^2 or sum g y_d y_e from
            // the moments shifted by the current mean c
            const double* Rm = mrec.data() + ((size_t)m * NP + j) * KS;
            const float* c = mvc.data() + ((size_t)m * NP + j) * KM;
            const double Wm = Rm[0];
            q[0] = Wm;
            for (int d = 0; d < D; ++d) q[1 + d] = Rm[1 + d] + c[d] * Wm;
            if (fam == HMM_DIAG_GAUSS) {
              for (int d = 0; d < D; ++d)
                q[1 + D + d] = Rm[1 + D + d] + 2.0 * c[d] * Rm[1 + d] + (double)c[d] * c[d] * Wm;
            } else {
              for (int d = 0; d < D; ++d)
                for (int e = 0; e < D; ++e)
                  q[1 + D + d * D + e] = Rm[1 + D + d * D + e] + c[d] * Rm[1 + e] + c[e] * Rm[1 + d] +
                                         (double)c[d] * c[e] * Wm;
            }
            break;
          }
          default:
            for (int z = 0; z < canon_fam_count(fam, md->dim_arg); ++z) q[z] = 0.0;
            q[0] = W;
            break;
        }
        q += canon_fam_count(fam, md->dim_arg);
      }
    }
  });
}

hmm_status hmm_stats_device_buffer(hmm_stats stats, double** d_values, int64_t* n_values) {
  return guarded([&] {
    HMM_REQUIRE(stats && d_values && n_values, "NULL argument");
    *d_values = stats->rec.as<double>();
    *n_values = (int64_t)stats->model->M * rec_size(stats->model->NP);
  });
}

hmm_status hmm_stats_set_allreduce(hmm_stats stats, hmm_allreduce_fn fn, void* user) {
  return guarded([&] {
    HMM_REQUIRE(stats != nullptr, "stats is NULL");
    stats->reduce_fn = fn;
    stats->reduce_user = fn ? user : nullptr;
  });
}

hmm_status hmm_stats_record(hmm_stats stats, int32_t index, void** d_values, int64_t* n_values, int32_t* op) {
  return guarded([&] {
    HMM_REQUIRE(stats && d_values && n_values && op, "NULL argument");
    int o = 0;
    record_view(stats, index, d_values, n_values, &o);
    *op = o;
  });
}

hmm_status hmm_estep_stats(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, hmm_stats stats,
                           double* d_loglik, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && stats, "NULL argument");
    HMM_REQUIRE(stats->model == model, "stats belong to another model");
    check_batch(model, batch);
    if (batch->n_seq == 0) {
      zero_stats(model, stats, S(stream));
    } else {
      PlanRef pr;
      get_plan(ctx, model, batch, S(stream), pr);
      run_estep(ctx, model, batch, pr.p, nullptr, nullptr, d_loglik, true, stats, S(stream));
      if (pr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
    }
    for (int i = 0; i < 3; ++i) {   // combine the shards' records
      void* p = nullptr;
      int64_t n = 0;
      int op = 0;
      record_view(stats, i, &p, &n, &op);
      call_reduce(stats, p, n, op, S(stream));
    }
  });
}

hmm_status hmm_mstep(hmm_ctx ctx, hmm_model model, hmm_stats stats, const hmm_batch* batch,
                     const hmm_mstep_opts* opts, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && stats, "NULL argument");
    HMM_REQUIRE(stats->model == model, "stats belong to another model");
    HMM_REQUIRE(stats->valid, "statistics were never computed");
    PlanRef pr;
    if (batch && (model->any_negbin || model->any_weibull)) {
      check_batch(model, batch);
      if (batch->n_seq > 0) get_plan(ctx, model, batch, S(stream), pr);
    }
    run_mstep(ctx, model, stats, to_opts(opts), batch, pr.p, S(stream));
    if (pr.owned) HMM_CUDA(cudaStreamSynchronize(S(stream)));
  });
}

hmm_status hmm_fit(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, const hmm_fit_opts* opts,
                   double* h_loglik_trace, int32_t* iters_done, void* stream) {
  return guarded([&] {
    HMM_REQUIRE(ctx && model && opts, "NULL argument");
    HMM_REQUIRE(opts->max_iter >= 0, "max_iter must be >= 0");
    check_batch(model, batch);
    // The iterations run on the context's own non-blocking stream (a graph
    // cannot be captured on the legacy default stream); the caller's stream
    // is drained first and the call returns after the loop has finished.
    HMM_CUDA(cudaStreamSynchronize(S(stream)));
    cudaStream_t st = ctx->work_stream;
    PlanRef pr;
    get_plan(ctx, model, batch, st, pr);
    hmm_stats stats = nullptr;
    hmm_status s0 = hmm_stats_create(ctx, model, &stats);
    if (s0 != HMM_OK) throw Error{s0, hmm_last_error()};
    struct StatsGuard {
      hmm_stats s;
      ~StatsGuard() { hmm_stats_destroy(s); }
    } sg{stats};
    const MStepOpts mo = to_opts(&opts->mstep);
    const int M = model->M, RS = rec_size(model->NP);
    const int iters = opts->max_iter;
    ctx->trace.ensure((size_t)std::max(iters, 1) * M * 8 + 64);
    int* it_dev = reinterpret_cast<int*>(ctx->trace.as<char>() + (size_t)std::max(iters, 1) * M * 8);
    HMM_CUDA(cudaMemsetAsync(it_dev, 0, sizeof(int), st));
    if (!pr.owned && pr.p->estep_G == 0 && iters >= 3 && model->NP <= 32) {
      hmm_status ts = hmm_plan_autotune(ctx, model, batch, nullptr, st);
      if (ts != HMM_OK) throw Error{ts, hmm_last_error()};
    }
    // make every buffer the iteration needs exist before any capture
    run_estep(ctx, model, batch, pr.p, nullptr, nullptr, nullptr, true, stats, st);
    prepare_mstep(model, stats, batch, pr.p);
    HMM_CUDA(cudaStreamSynchronize(st));
    const bool viterbi_training = opts->trainer == 1;
    HMM_REQUIRE(opts->trainer == 0 || opts->trainer == 1, "trainer must be 0 (Baum-Welch) or 1 (Viterbi)");
    if (viterbi_training) {   // size the Viterbi-training buffers before any capture
      run_estep_viterbi(ctx, model, batch, pr.p, stats, nullptr, st);
      HMM_CUDA(cudaStreamSynchronize(st));
    }
    auto one_iter = [&]() {
      if (viterbi_training)
        run_estep_viterbi(ctx, model, batch, pr.p, stats, nullptr, st);
      else
        run_estep(ctx, model, batch, pr.p, nullptr, nullptr, nullptr, true, stats, st);
      trace_gather_kernel<<<(M + 255) / 256, 256, 0, st>>>(stats->rec.as<double>(), RS, M,
                                                          ctx->trace.as<double>(), it_dev);
      HMM_CUDA(cudaGetLastError());
      run_mstep(ctx, model, stats, mo, batch, pr.p, st);
      bump_kernel<<<1, 1, 0, st>>>(it_dev);
      HMM_CUDA(cudaGetLastError());
    };
    int done = 0;
    if (opts->tol <= 0.0 && iters > 0) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      HMM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      try {
        one_iter();
      } catch (...) {
        cudaStreamEndCapture(st, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      HMM_CUDA(cudaStreamEndCapture(st, &graph));
      cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) throw Error{HMM_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)};
      for (int k = 0; k < iters; ++k) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) break;
      }
      cudaGraphExecDestroy(exec);
      if (e != cudaSuccess) throw Error{HMM_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e)};
      done = iters;
    } else {
      double prev = 0.0;
      std::vector<double> row(M);
      for (int k = 0; k < iters; ++k) {
        one_iter();
        ++done;
        HMM_CUDA(cudaMemcpyAsync(row.data(), ctx->trace.as<double>() + (size_t)k * M, M * 8,
                                 cudaMemcpyDeviceToHost, st));
        HMM_CUDA(cudaStreamSynchronize(st));
        double tot = 0.0;
        for (double v : row) tot += v;
        if (k > 0 && std::fabs(tot - prev) <= opts->tol * std::fabs(tot)) break;
        prev = tot;
      }
    }
    if (h_loglik_trace && done > 0) {
      HMM_CUDA(cudaMemcpyAsync(h_loglik_trace, ctx->trace.p, (size_t)done * M * 8, cudaMemcpyDeviceToHost, st));
    }
    HMM_CUDA(cudaStreamSynchronize(st));
    if (iters_done) *iters_done = done;
  });
}

}  // extern "C"
