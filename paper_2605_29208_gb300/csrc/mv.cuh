// Multivariate emission families of paper Sec. 4.5: diagonal Gaussian
// (Eq. 20-21) and full-covariance Gaussian (Eq. 22-24).
//
// Emissions are evaluated into a float32 log b table that the fused E-step
// and Viterbi kernels read (table mode).  Derived per-state tables (float32):
//   diagonal: mu[D], h[D] = 1 / (2 var), c = -1/2 sum_d log(2 pi var_d)
//   full:     mu[D], Linv[D][D] (inverse of the Cholesky factor of Sigma,
//             lower triangular), c = -D/2 log 2 pi - sum_d log L_dd
// so log b = c - sum_d h_d (y_d - mu_d)^2  or  c - 1/2 |Linv (y - mu)|^2.
// The statistics are shifted moments around the current mean (float32
// per sequence, two-level), reduced in fixed order in float64; the M-step
// recovers mu = shift + S1 / W and the (co)variance, adds eps I (Sec. 4.5)
// and refactors.
#pragma once

#include "common.cuh"
#include "mstep_types.h"

namespace hmm {

__host__ __device__ inline int mv_coef_count(int fam, int D) {
  return fam == HMM_DIAG_GAUSS ? 2 * D + 1 : D + D * D + 1;
}
// statistic slots per state: W, S1[D], then S2[D] (diagonal) or S2[D][D] (full)
__host__ __device__ inline int mv_stat_count(int fam, int D) {
  return fam == HMM_DIAG_GAUSS ? 1 + 2 * D : 1 + D + D * D;
}

// Derived tables of one (model, state) from theta (float64, device).
__device__ inline void mv_derive_state(int fam, int D, const double* th, float* c) {
  constexpr double L2PI = 1.83787706640934548356;   // log(2 pi)
  if (fam == HMM_DIAG_GAUSS) {
    double cc = 0.0;
    for (int d = 0; d < D; ++d) {
      const double mu = th[d], var = th[D + d];
      c[d] = (float)mu;
      c[D + d] = (float)(0.5 / var);
      cc += -0.5 * (L2PI + log(var));
    }
    c[2 * D] = (float)cc;
    return;
  }
  // full covariance: Cholesky Sigma = L L^T (float64), then Linv
  double L[32 * 32], Li[32 * 32];
  const double* S = th + D;
  bool ok = D <= 32;
  for (int i = 0; i < D && ok; ++i)
    for (int j = 0; j <= i; ++j) {
      double acc = S[i * D + j];
      for (int k = 0; k < j; ++k) acc -= L[i * D + k] * L[j * D + k];
      if (i == j) {
        if (!(acc > 0.0)) {
          ok = false;
          break;
        }
        L[i * D + i] = sqrt(acc);
      } else {
        L[i * D + j] = acc / L[j * D + j];
      }
    }
  for (int d = 0; d < D; ++d) c[d] = (float)th[d];
  if (!ok) {   // not positive definite: density 0 everywhere
    for (int z = 0; z < D * D; ++z) c[D + z] = 0.f;
    c[D + D * D] = -INFINITY;
    return;
  }
  double logdet = 0.0;
  for (int i = 0; i < D; ++i) logdet += log(L[i * D + i]);
  for (int i = 0; i < D; ++i) {
    for (int j = 0; j < D; ++j) Li[i * D + j] = 0.0;
    Li[i * D + i] = 1.0 / L[i * D + i];
    for (int j = 0; j < i; ++j) {
      double acc = 0.0;
      for (int k = j; k < i; ++k) acc += L[i * D + k] * Li[k * D + j];
      Li[i * D + j] = -acc / L[i * D + i];
    }
  }
  bool rep = true;   // the inverse factor must fit float32
  for (int z = 0; z < D * D; ++z) rep = rep && fabs(Li[z]) < 1e30;
  if (!rep) {
    for (int z = 0; z < D * D; ++z) c[D + z] = 0.f;
    c[D + D * D] = -INFINITY;
    return;
  }
  for (int z = 0; z < D * D; ++z) c[D + z] = (float)Li[z];
  c[D + D * D] = (float)(-0.5 * D * L2PI - logdet);
}

__global__ void mv_derive_kernel(const int* __restrict__ family, const double* __restrict__ theta, int M, int NP,
                                 int N, int P, int D, int KM, float* __restrict__ mvc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  const int m = idx / NP, k = idx % NP;
  const int fam = family[m];
  float* c = mvc + (size_t)idx * KM;
  if (k >= N) {                      // padding state: log b = -inf
    for (int z = 0; z < KM; ++z) c[z] = 0.f;
    c[mv_coef_count(fam, D) - 1] = -INFINITY;
    return;
  }
  mv_derive_state(fam, D, theta + (size_t)idx * P, c);
}

// log b_j(y_t) (natural log) for every row of the batch: one block per
// (sequence, tile of 32 rows); threads stride over (row, state).
__global__ void mv_emission_kernel(const int* __restrict__ family, const float* __restrict__ mvc, int NP, int N,
                                   int D, int KM, const float* __restrict__ y, const int64_t* __restrict__ offsets,
                                   const int32_t* __restrict__ model_id, const int32_t* __restrict__ tile_seq,
                                   const int32_t* __restrict__ tile_row, float* __restrict__ logb) {
  extern __shared__ float ys[];       // [32][D]
  const int s = tile_seq[blockIdx.x];
  const int64_t r0 = offsets[s] + tile_row[blockIdx.x];
  const int64_t r1 = min(r0 + 32, offsets[s + 1]);
  const int nr = (int)(r1 - r0);
  const int m = model_id[s];
  const int fam = family[m];
  for (int z = threadIdx.x; z < nr * D; z += blockDim.x) ys[z] = y[r0 * D + z];
  __syncthreads();
  for (int z = threadIdx.x; z < nr * N; z += blockDim.x) {
    const int r = z / N, k = z % N;
    const float* c = mvc + ((size_t)m * NP + k) * KM;
    const float* yr = ys + r * D;
    float q = 0.f;
    if (fam == HMM_DIAG_GAUSS) {
      for (int d = 0; d < D; ++d) {
        const float e = yr[d] - c[d];
        q = fmaf(c[D + d] * e, e, q);
      }
      logb[(r0 + r) * N + k] = c[2 * D] - q;
    } else {
      const float* Li = c + D;
      for (int i = 0; i < D; ++i) {
        float zi = 0.f;
        for (int j = 0; j <= i; ++j) zi = fmaf(Li[i * D + j], yr[j] - c[j], zi);
        q = fmaf(zi, zi, q);
      }
      logb[(r0 + r) * N + k] = c[D + D * D] - 0.5f * q;
    }
  }
}

// Shifted weighted moments per sequence and state from the occupancies:
// part[s][k][*] = W, sum g (y - mu), then sum g (y-mu)_d^2 (diagonal) or
// sum g (y-mu)(y-mu)^T (full).  One block per sequence, one thread per
// (state, slot); two-level float32 sums over t.
__global__ void mv_stats_kernel(const int* __restrict__ family, const float* __restrict__ mvc, int NP, int N, int D,
                                int KM, int KS, const float* __restrict__ y, const float* __restrict__ gamma,
                                const int64_t* __restrict__ offsets, const int32_t* __restrict__ model_id,
                                float* __restrict__ part) {
  const int s = blockIdx.x;
  const int64_t b = offsets[s], e = offsets[s + 1];
  const int m = model_id[s];
  const int fam = family[m];
  const int total = NP * KS;
  for (int f = threadIdx.x; f < total; f += blockDim.x) {
    const int k = f / KS, z = f % KS;
    float a = 0.f;
    if (k < N && z < mv_stat_count(fam, D)) {   // a set mixing both families pads the diagonal records
      const float* c = mvc + ((size_t)m * NP + k) * KM;
      int d1 = -1, d2 = -1;
      if (z >= 1 && z <= D) d1 = z - 1;
      else if (z > D) {
        if (fam == HMM_DIAG_GAUSS) d1 = d2 = z - 1 - D;
        else {
          d1 = (z - 1 - D) / D;
          d2 = (z - 1 - D) % D;
        }
      }
      const float mu1 = d1 >= 0 ? c[d1] : 0.f, mu2 = d2 >= 0 ? c[d2] : 0.f;
      float in = 0.f;
      int cnt = 0;
      for (int64_t t = b; t < e; ++t) {
        const float g = gamma[t * N + k];
        float v = g;
        if (d1 >= 0) v *= y[t * D + d1] - mu1;
        if (d2 >= 0) v *= y[t * D + d2] - mu2;
        in += v;
        if (++cnt == 64) {
          a += in;
          in = 0.f;
          cnt = 0;
        }
      }
      a += in;
    }
    part[(size_t)s * total + f] = a;
  }
}

// M-step of the multivariate families (one thread per (model, state)).
__global__ void mv_mstep_kernel(const int* __restrict__ family, double* __restrict__ theta, const float* __restrict__ mvc,
                                const double* __restrict__ rec, int M, int NP, int N, int P, int D, int KM, int KS,
                                double collapse_eps, double tikhonov_eps) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  const int m = idx / NP, k = idx % NP;
  if (k >= N) return;
  const int fam = family[m];
  if (fam != HMM_DIAG_GAUSS && fam != HMM_FULL_GAUSS) return;
  const double* R = rec + (size_t)idx * KS;
  const float* c = mvc + (size_t)idx * KM;
  double* th = theta + (size_t)idx * P;
  const double W = R[0];
  if (W < collapse_eps) return;                        // Sec. 4.4
  double nt[32 + 32 * 32];
  bool ok = true;
  for (int d = 0; d < D; ++d) {
    nt[d] = (double)c[d] + R[1 + d] / W;
    ok = ok && isfinite(nt[d]);
  }
  if (fam == HMM_DIAG_GAUSS) {                         // Eq. 21
    for (int d = 0; d < D; ++d) {
      const double m1 = R[1 + d] / W;
      nt[D + d] = R[1 + D + d] / W - m1 * m1;
      ok = ok && isfinite(nt[D + d]) && nt[D + d] > 0.0;
    }
  } else {                                             // Eq. 23-24
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        const double mi = R[1 + i] / W, mj = R[1 + j] / W;
        const double cij = 0.5 * (R[1 + D + i * D + j] + R[1 + D + j * D + i]) / W - mi * mj;
        nt[D + i * D + j] = cij + (i == j ? tikhonov_eps : 0.0);
      }
    // positive definite (float64 Cholesky), else the update is undefined
    double L[32 * 32];
    for (int i = 0; i < D && ok; ++i)
      for (int j = 0; j <= i && ok; ++j) {
        double acc = nt[D + i * D + j];
        for (int k2 = 0; k2 < j; ++k2) acc -= L[i * D + k2] * L[j * D + k2];
        if (i == j) {
          ok = isfinite(acc) && acc > 0.0;
          if (ok) L[i * D + i] = sqrt(acc);
        } else {
          L[i * D + j] = acc / L[j * D + j];
        }
      }
  }
  // an undefined update keeps theta_j (the collapse guard of Sec. 4.4)
  if (ok)
    for (int z = 0; z < mv_coef_count(fam, D) - 1; ++z) th[z] = nt[z];
}

}  // namespace hmm

namespace hmm {

// Large-N statistics of the multivariate families: raw weighted moments
// R[j][z] = sum_t gamma_t(j) f_z(y_t) per 64-sequence chunk with
// f = (1, y_d, y_d^2) (diagonal) or (1, y_d, y_d y_e) (full), as a
// 64-state x 64-feature tiled outer-product sum over the chunk's rows
// (float32 in registers, float64 every 256 rows); mv_shift_kernel turns the
// reduced sums into the moments about the current mean that mv_mstep_kernel
// reads.
constexpr int MVM_TILE = 64;
constexpr int MVM_KT = 16;

__device__ __forceinline__ float mv_feature(int fam, int D, int z, const float* yr) {
  if (fam == HMM_DISCRETE) return yr[0] == (float)z ? 1.f : 0.f;   // symbol indicator 1[y = z]
  if (is_ext_family(fam)) return ext_feature(fam, z, yr[0]);
  if (z == 0) return 1.f;
  if (z <= D) return yr[z - 1];
  const int q = z - 1 - D;
  if (fam == HMM_DIAG_GAUSS) return q < D ? yr[q] * yr[q] : 0.f;
  return q < D * D ? yr[q / D] * yr[q % D] : 0.f;
}

// Block (tile, c, z): rows [z per, (z + 1) per) of chunk c's rows taken in
// seq_by_model order (crow[q] = the chunk rows before position q), in slabs
// of MVM_KT rows; the next slab's values are loaded into registers while the
// current one is accumulated (double-buffered shared memory, one barrier per
// slab).  part[(c split + z)][NP][KS] float64; mv_split_combine_kernel adds
// the splits of a chunk in order.
__global__ void __launch_bounds__(256) mv_moments_kernel(const int* __restrict__ family, int NP, int N, int D, int KS,
                                                         const float* __restrict__ y, const float* __restrict__ gamma,
                                                         const int64_t* __restrict__ offsets,
                                                         const int32_t* __restrict__ model_id,
                                                         const int32_t* __restrict__ seq_by_model,
                                                         const int32_t* __restrict__ chunk_lo,
                                                         const int32_t* __restrict__ chunk_hi,
                                                         const int64_t* __restrict__ crow, int split,
                                                         double* __restrict__ part) {
  __shared__ __align__(16) float Xs[2][MVM_KT][MVM_TILE];
  __shared__ __align__(16) float Fs[2][MVM_KT][MVM_TILE];
  const int ftiles = (KS + MVM_TILE - 1) / MVM_TILE;
  const int ti = blockIdx.x / ftiles, tf = blockIdx.x % ftiles;
  const int c = blockIdx.y, zsp = blockIdx.z;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int lo = chunk_lo[c], hi = chunk_hi[c];
  const int fam = family[model_id[seq_by_model[lo]]];
  const int nf = fam == HMM_DISCRETE ? KS : (is_ext_family(fam) ? ext_stat_count(fam) : mv_stat_count(fam, D));
  const int slast = seq_by_model[hi - 1];
  const int64_t rows = crow[hi - 1] + (offsets[slast + 1] - offsets[slast]);
  const int64_t per = (rows + split - 1) / split;
  const int64_t r0 = (int64_t)zsp * per < rows ? (int64_t)zsp * per : rows, r1 = r0 + per < rows ? r0 + per : rows;
  float acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f, dacc[p][q] = 0.0;
  int since = 0, buf = 0;
  constexpr int PER_T = MVM_KT * MVM_TILE / 256;   // slab entries per thread
  for (int qs = lo; qs < hi && r0 < r1; ++qs) {
    const int s = seq_by_model[qs];
    const int64_t b = offsets[s], len = offsets[s + 1] - b, cs = crow[qs];
    const int64_t ta = r0 - cs > 0 ? r0 - cs : 0, tb = r1 - cs < len ? r1 - cs : len;
    if (ta >= tb) continue;
    float px[PER_T], pf[PER_T];
    auto fetch = [&](int64_t t0) {
#pragma unroll
      for (int e = 0; e < PER_T; ++e) {
        const int z = tid + 256 * e, r = z / MVM_TILE, col = z % MVM_TILE;
        const int64_t t = t0 + r;
        float xv = 0.f, fv = 0.f;
        if (t < tb) {
          const int j = ti * MVM_TILE + col, f = tf * MVM_TILE + col;
          if (j < N) xv = gamma[(b + t) * N + j];
          if (f < nf) fv = mv_feature(fam, D, f, y + (b + t) * D);
        }
        px[e] = xv;
        pf[e] = fv;
      }
    };
    fetch(ta);
    for (int64_t t0 = ta; t0 < tb; t0 += MVM_KT) {
#pragma unroll
      for (int e = 0; e < PER_T; ++e) {
        const int z = tid + 256 * e, r = z / MVM_TILE, col = z % MVM_TILE;
        Xs[buf][r][col] = px[e];
        Fs[buf][r][col] = pf[e];
      }
      if (t0 + MVM_KT < tb) fetch(t0 + MVM_KT);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < MVM_KT; ++r) {
        const float4 x = *reinterpret_cast<const float4*>(&Xs[buf][r][ty * 4]);
        const float4 f4 = *reinterpret_cast<const float4*>(&Fs[buf][r][tx * 4]);
        const float xa[4] = {x.x, x.y, x.z, x.w}, fa[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(xa[p], fa[q], acc[p][q]);
      }
      buf ^= 1;
      since += MVM_KT;
      if (since >= 256) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) dacc[p][q] += acc[p][q], acc[p][q] = 0.f;
        since = 0;
      }
    }
  }
  double* o = part + ((size_t)c * split + zsp) * NP * KS;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = ti * MVM_TILE + ty * 4 + p, f = tf * MVM_TILE + tx * 4 + q;
      if (j < NP && f < KS) o[(size_t)j * KS + f] = dacc[p][q] + (double)acc[p][q];
    }
}

// out[c][e] = sum over z = 0, 1, .. of part[c split + z][e] (fixed order)
__global__ void mv_split_combine_kernel(const double* __restrict__ part, int split, int64_t rec,
                                        double* __restrict__ out) {
  const int c = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rec; e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < split; ++z) v += part[((size_t)c * split + z) * rec + e];
    out[(size_t)c * rec + e] = v;
  }
}

// Raw feature sums per sequence for padded N <= 32 and few features
// (discrete with K <= FEAT_SMALL_MAX symbols, the log-normal .. Pareto
// group): part[s][k][z] = sum_t gamma_t(k) f_z(y_t).  One block of 256
// threads per sequence; a warp covers 32 / NP rows per pass with one lane
// per (row, state), so each pass reads whole occupancy rows; a thread keeps
// one float32 sum per feature (flushed every 64 passes), and the partials of
// a state are added in a fixed (warp, row-in-warp) order, so the result does
// not depend on scheduling.  The per-sequence records are then reduced like
// the multivariate moments (chunks, then models).
constexpr int FEAT_SMALL_MAX = 8;

__global__ void __launch_bounds__(256) feat_stats_kernel(const int* __restrict__ family, int NP, int N, int KS,
                                                         const float* __restrict__ y,
                                                         const float* __restrict__ gamma,
                                                         const int64_t* __restrict__ offsets,
                                                         const int32_t* __restrict__ model_id,
                                                         float* __restrict__ part) {
  __shared__ float red[FEAT_SMALL_MAX][256];
  const int s = blockIdx.x;
  const int64_t b = offsets[s], e = offsets[s + 1];
  const int fam = family[model_id[s]];
  const int nf = fam == HMM_DISCRETE ? KS : ext_stat_count(fam);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int RW = 32 / NP;                       // rows per warp and pass
  const int k = lane % NP, rs = lane / NP;
  float acc[FEAT_SMALL_MAX], in[FEAT_SMALL_MAX];
#pragma unroll
  for (int z = 0; z < FEAT_SMALL_MAX; ++z) acc[z] = in[z] = 0.f;
  int cnt = 0;
  for (int64_t t = b + (int64_t)w * RW + rs; t < e; t += (int64_t)nw * RW) {
    if (k < N) {
      const float g = gamma[t * N + k];
#pragma unroll
      for (int z = 0; z < FEAT_SMALL_MAX; ++z)
        if (z < nf) in[z] = fmaf(g, mv_feature(fam, 1, z, y + t), in[z]);
    }
    if (++cnt == 64) {
#pragma unroll
      for (int z = 0; z < FEAT_SMALL_MAX; ++z) acc[z] += in[z], in[z] = 0.f;
      cnt = 0;
    }
  }
#pragma unroll
  for (int z = 0; z < FEAT_SMALL_MAX; ++z) red[z][threadIdx.x] = acc[z] + in[z];
  __syncthreads();
  // state k's partials sit at threads w * 32 + r * NP + k
  for (int f = threadIdx.x; f < NP * KS; f += blockDim.x) {
    const int kk = f / KS, z = f % KS;
    float v = 0.f;
    if (kk < N && z < nf)
      for (int ww = 0; ww < nw; ++ww)
        for (int r = 0; r < RW; ++r) v += red[z][ww * 32 + r * NP + kk];
    part[(size_t)s * NP * KS + f] = v;
  }
}

// Raw moments -> moments about the current (float32) mean, in place.
__global__ void mv_shift_kernel(const int* __restrict__ family, const float* __restrict__ mvc, int M, int NP, int N,
                                int D, int KM, int KS, double* __restrict__ rec) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  const int m = idx / NP, k = idx % NP;
  if (k >= N) return;
  const int fam = family[m];
  double* R = rec + (size_t)idx * KS;
  const float* c = mvc + (size_t)idx * KM;
  const double W = R[0];
  if (fam == HMM_DIAG_GAUSS) {
    for (int d = 0; d < D; ++d) {
      const double mu = c[d], m1 = R[1 + d];
      R[1 + D + d] = R[1 + D + d] - 2.0 * mu * m1 + mu * mu * W;
      R[1 + d] = m1 - mu * W;
    }
  } else {
    for (int d = 0; d < D; ++d)
      for (int e = 0; e < D; ++e) {
        const double md = c[d], me = c[e];
        R[1 + D + d * D + e] = R[1 + D + d * D + e] - md * R[1 + e] - me * R[1 + d] + md * me * W;
      }
    for (int d = 0; d < D; ++d) R[1 + d] -= (double)c[d] * W;
  }
}

}  // namespace hmm

namespace hmm {

// Tiled form of mv_emission_kernel: a block computes one 32-row tile of a
// sequence for 64 states, with the rows and the states' tables staged in
// shared memory; a thread owns 2 rows x 4 states.  Diagonal Gaussian for any
// D <= 32, full covariance for D <= MV_TILED_FULL_D (the triangular solve
// keeps the D differences of a (row, state) pair in registers).
constexpr int MV_TILED_FULL_D = 16;

template <int FAM>
__global__ void __launch_bounds__(256) mv_emission_tiled_kernel(const float* __restrict__ mvc, int NP, int N, int D,
                                                                int KM, const float* __restrict__ y,
                                                                const int64_t* __restrict__ offsets,
                                                                const int32_t* __restrict__ model_id,
                                                                const int32_t* __restrict__ tile_seq,
                                                                const int32_t* __restrict__ tile_row,
                                                                float* __restrict__ logb) {
  extern __shared__ float msm[];
  const int KMP = KM | 1;                  // odd stride: state rows on different banks
  float* ys = msm;                         // [32][D + 1]
  float* cs = ys + 32 * (D + 1);           // [64][KMP]
  const int s = tile_seq[blockIdx.x];
  const int64_t r0 = offsets[s] + tile_row[blockIdx.x];
  const int nr = (int)min((int64_t)32, offsets[s + 1] - r0);
  const int m = model_id[s];
  const int k0 = blockIdx.y * 64;
  const int nk = min(64, N - k0);
  for (int z = threadIdx.x; z < nr * D; z += blockDim.x) ys[(z / D) * (D + 1) + z % D] = y[r0 * D + z];
  for (int z = threadIdx.x; z < nk * KM; z += blockDim.x)
    cs[(z / KM) * KMP + z % KM] = mvc[((size_t)m * NP + k0 + z / KM) * KM + z % KM];
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int ra = ty * 2;
  float acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
  if constexpr (FAM == HMM_DIAG_GAUSS) {
    for (int d = 0; d < D; ++d) {
      const float y0 = ys[ra * (D + 1) + d], y1 = ys[(ra + 1) * (D + 1) + d];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* c = cs + (tx * 4 + q) * KMP;
        const float mu = c[d], h = c[D + d];
        const float e0 = y0 - mu, e1 = y1 - mu;
        acc[0][q] = fmaf(h * e0, e0, acc[0][q]);
        acc[1][q] = fmaf(h * e1, e1, acc[1][q]);
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float* yr = ys + (ra + a) * (D + 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* c = cs + (tx * 4 + q) * KMP;
        float e[MV_TILED_FULL_D];
#pragma unroll
        for (int j = 0; j < MV_TILED_FULL_D; ++j) e[j] = j < D ? yr[j] - c[j] : 0.f;
        const float* Li = c + D;
        float qq = 0.f;
#pragma unroll
        for (int i = 0; i < MV_TILED_FULL_D; ++i) {
          if (i >= D) break;
          float zi = 0.f;
#pragma unroll
          for (int j = 0; j <= i; ++j) zi = fmaf(Li[i * D + j], e[j], zi);
          qq = fmaf(zi, zi, qq);
        }
        acc[a][q] = qq;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (ra + a >= nr) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = tx * 4 + q;
      if (k >= nk) continue;
      const float* c = cs + k * KMP;
      const float cst = FAM == HMM_DIAG_GAUSS ? c[2 * D] : c[D + D * D];
      logb[(r0 + ra + a) * N + k0 + k] = FAM == HMM_DIAG_GAUSS ? cst - acc[a][q] : cst - 0.5f * acc[a][q];
    }
  }
}

}  // namespace hmm

namespace hmm {

// ---------------------------------------------------------------------------
// Discrete (categorical) family (Sec. 4, "Discrete"): per state K symbol
// probabilities; log b_j(y) = ln p_jy for an integer y in [0, K), else -inf.
// ---------------------------------------------------------------------------
__global__ void discrete_derive_kernel(const double* __restrict__ theta, int M, int NP, int N, int P, int K,
                                       float* __restrict__ dtab) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  const int k = idx % NP;
  float* t = dtab + (size_t)idx * K;
  const double* th = theta + (size_t)idx * P;
  for (int z = 0; z < K; ++z) t[z] = (k < N && th[z] > 0.0) ? (float)log(th[z]) : -INFINITY;
}

// log b table [total_T][N]: blocks (sequence, slab of EMIS_SLAB rows),
// threads over (t, state)
__global__ void discrete_emission_kernel(const float* __restrict__ dtab, int NP, int N, int K,
                                         const float* __restrict__ y, const int64_t* __restrict__ offsets,
                                         const int32_t* __restrict__ model_id, float* __restrict__ logb) {
  const int s = blockIdx.x;
  const int64_t b = offsets[s] + (int64_t)blockIdx.y * EMIS_SLAB;
  const int64_t e = min(offsets[s + 1], b + (int64_t)EMIS_SLAB);
  if (b >= e) return;
  const int m = model_id[s];
  const float* tab = dtab + (size_t)m * NP * K;
  if (N <= (int)blockDim.x) {   // a fixed (row, state) slot per thread, as in emission_kernel
    const int rpp = blockDim.x / N, rr = threadIdx.x / N, j = threadIdx.x % N;
    if (rr >= rpp) return;
    const float* tj = tab + (size_t)j * K;
    for (int64_t t = b + rr; t < e; t += rpp) {
      const float v = y[t];
      const bool ok = v >= 0.f && v < (float)K && floorf(v) == v;
      logb[t * N + j] = ok ? tj[(int)v] : -INFINITY;
    }
    return;
  }
  for (int64_t idx = threadIdx.x; idx < (e - b) * N; idx += blockDim.x) {
    const int64_t t = b + idx / N;
    const int j = (int)(idx % N);
    const float v = y[t];
    const bool ok = v >= 0.f && v < (float)K && floorf(v) == v;
    logb[t * N + j] = ok ? tab[(size_t)j * K + (int)v] : -INFINITY;
  }
}

// p_jk = count_jk / sum_k count_jk (Sec. 4, "Discrete"); a state whose
// weight is below the collapse threshold keeps its probabilities (Sec. 4.4)
__global__ void discrete_mstep_kernel(double* __restrict__ theta, const double* __restrict__ rec, int M, int NP, int N,
                                      int P, int K, double collapse_eps) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  if (idx % NP >= N) return;
  const double* R = rec + (size_t)idx * K;
  double W = 0.0;
  for (int z = 0; z < K; ++z) W += R[z];
  if (!(W >= collapse_eps)) return;
  double* th = theta + (size_t)idx * P;
  for (int z = 0; z < K; ++z) th[z] = R[z] / W;
}

}  // namespace hmm

