// The plain float32 log-space path: the recursions of paper Sec. 3.2 written
// directly, with a full log-sum-exp (N exponentials per state and step) and
// raw log-space alpha-hat / beta-hat stored in float32 (log2 units), then a
// posterior pass with N^2 exponentials per step for xi.  It is the reference
// GPU implementation that the fused kernels are measured against; its
// statistics use the same per-sequence partial layout (forward slot) so the
// same reductions and M-step follow.
//
// Layout: one lane per state, NP lanes per sequence (NP <= 32), several
// sequences per warp; alpha / beta rows are exchanged through shared memory.
#pragma once

#include "common.cuh"
#include "estep_small.cuh"

namespace hmm {

struct PlainArgs {
  const float* y;
  const int64_t* offsets;
  const int32_t* model_id;
  int32_t n_seq;
  ModelView mv;
  float* alpha;       // [total_T][NP] log2 alpha-hat
  float* beta;        // [total_T][NP] log2 beta-hat
  float* partials;    // [S][2][NP][NP + NST]
  double* loglik;     // [S]
  float* gamma;       // [total_T][N] occupancies, or nullptr (kept for the data-pass M-steps)
};

// lse in base 2 over i of x[i] + c[i]
template <int NP>
__device__ __forceinline__ float lse2_plain(const float* x, const float* c) {
  float m = -INFINITY;
#pragma unroll
  for (int i = 0; i < NP; ++i) m = fmaxf(m, x[i] + c[i]);
  if (m == -INFINITY) return -INFINITY;
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NP; ++i) s += ex2f(x[i] + c[i] - m);
  return m + log2f(s);
}

template <int NP>
__global__ void __launch_bounds__(128) plain_recursions_kernel(PlainArgs a) {
  constexpr int SPW = 32 / NP;
  __shared__ float xb[4][SPW][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / NP, j = lane % NP;
  const int s = (blockIdx.x * 4 + w) * SPW + grp;
  const bool valid = s < a.n_seq;
  const int64_t base = valid ? a.offsets[s] : 0;
  const int T = valid ? (int)(a.offsets[s + 1] - base) : 0;
  const int m = valid ? a.model_id[s] : 0;
  const int fam = a.mv.family[m];
  const int N = a.mv.N;
  float colA[NP], rowA[NP];
  for (int i = 0; i < NP; ++i) {
    colA[i] = a.mv.logA2[((size_t)m * NP + i) * NP + j];
    rowA[i] = a.mv.logA2[((size_t)m * NP + j) * NP + i];
  }
  float c[4];
  for (int z = 0; z < 4; ++z) c[z] = a.mv.coef[((size_t)m * NP + j) * KC + z];
  const float* nbt = a.mv.nbtab ? a.mv.nbtab + ((size_t)m * NP + j) * NB_YMAX : nullptr;
  int Tmax = T;
  for (int o = 16; o > 0; o >>= 1) Tmax = max(Tmax, __shfl_xor_sync(0xffffffffu, Tmax, o));
  auto emis = [&](int t) {
    const Feat f = feat_of(fam, a.y[base + t], a.mv.lfact2);
    return (f.ok && j < N) ? emis_log2(fam, f, c, nbt) : -INFINITY;
  };
  // forward (Eq. 1-2)
  float al = -INFINITY;
  for (int t = 0; t < Tmax; ++t) {
    const bool act = t < T;
    float x[NP];
    if (t > 0) {
      xb[w][grp][j] = al;
      __syncwarp();
      for (int i = 0; i < NP; ++i) x[i] = xb[w][grp][i];
      __syncwarp();
    }
    if (act) {
      const float lb = emis(t);
      al = (t == 0) ? a.mv.logpi2[(size_t)m * NP + j] + lb : lse2_plain<NP>(x, colA) + lb;
      a.alpha[(base + t) * NP + j] = al;
    }
  }
  // log-likelihood = lse_j alpha_T(j)
  xb[w][grp][j] = al;
  __syncwarp();
  if (valid && j == 0 && T > 0) {
    float x[NP], z[NP];
    for (int i = 0; i < NP; ++i) {
      x[i] = xb[w][grp][i];
      z[i] = 0.f;
    }
    a.loglik[s] = (double)lse2_plain<NP>(x, z) * kLn2;
  }
  if (valid && j == 0 && T == 0) a.loglik[s] = 0.0;
  __syncwarp();
  // backward: beta_T = 0, beta_t(i) = lse_j[log a_ij + log b_j(y_{t+1}) + beta_{t+1}(j)]
  float be = 0.f;
  for (int k = 0; k < Tmax; ++k) {
    const int t = T - 1 - k;
    const bool act = t >= 0;
    float x[NP];
    if (k > 0) {
      xb[w][grp][j] = act ? be + emis(t + 1) : -INFINITY;
      __syncwarp();
      for (int i = 0; i < NP; ++i) x[i] = xb[w][grp][i];
      __syncwarp();
    }
    if (act) {
      be = (k == 0) ? 0.f : lse2_plain<NP>(x, rowA);
      a.beta[(base + t) * NP + j] = be;
    }
  }
}

// gamma, xi (N^2 exponentials per step) and the family sums.
template <int NP>
__global__ void __launch_bounds__(128) plain_posterior_kernel(PlainArgs a) {
  constexpr int SPW = 32 / NP;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / NP, j = lane % NP;
  const int s = (blockIdx.x * 4 + w) * SPW + grp;
  if (s >= a.n_seq) return;
  const int64_t base = a.offsets[s];
  const int T = (int)(a.offsets[s + 1] - base);
  const int m = a.model_id[s];
  const int fam = a.mv.family[m];
  const int N = a.mv.N;
  float c[4], c2[2];
  for (int z = 0; z < 4; ++z) c[z] = a.mv.coef[((size_t)m * NP + j) * KC + z];
  c2[0] = a.mv.coef[((size_t)m * NP + j) * KC + 4];
  c2[1] = a.mv.coef[((size_t)m * NP + j) * KC + 5];
  const float* nbt = a.mv.nbtab ? a.mv.nbtab + ((size_t)m * NP + j) * NB_YMAX : nullptr;
  const float ll2 = T > 0 ? (float)(a.loglik[s] * kLog2e) : 0.f;
  float xi[NP], st[NST];
  for (int i = 0; i < NP; ++i) xi[i] = 0.f;
  for (int z = 0; z < NST; ++z) st[z] = 0.f;
  for (int t = 0; t < T; ++t) {
    const Feat f = feat_of(fam, a.y[base + t], a.mv.lfact2);
    const float* ar = a.alpha + (base + t) * NP;
    const float g = ex2f(ar[j] + a.beta[(base + t) * NP + j] - ll2);
    if (a.gamma && j < N) a.gamma[(base + t) * N + j] = g;
    st[0] += g;
    accumulate_stats(fam, f, c, c2, g, st);
    if (t == 0) st[NST - 1] += g;
    if (t + 1 < T) {
      // xi_t(i, j) without the a_ij factor: alpha_t(i) b_j(y_{t+1}) beta_{t+1}(j) / P
      const Feat f1 = feat_of(fam, a.y[base + t + 1], a.mv.lfact2);
      const float lb1 = (f1.ok && j < N) ? emis_log2(fam, f1, c, nbt) : -INFINITY;
      const float rj = lb1 + a.beta[(base + t + 1) * NP + j] - ll2;
      for (int i = 0; i < NP; ++i) xi[i] += ex2f(ar[i] + rj);
    }
  }
  float* p = a.partials + (((size_t)s * 2 + 0) * NP + j) * (NP + NST);
  for (int i = 0; i < NP; ++i) p[i] = xi[i];
  for (int z = 0; z < NST; ++z) p[NP + z] = st[z];
  float* q = a.partials + (((size_t)s * 2 + 1) * NP + j) * (NP + NST);
  for (int i = 0; i < NP + NST; ++i) q[i] = 0.f;
}

}  // namespace hmm
