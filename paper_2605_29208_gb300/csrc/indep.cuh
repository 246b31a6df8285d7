// Independent-components emissions (paper Sec. 4.5, "Independent
// components"): state j of model m emits y_t in R^D with density
//   b_j(y_t) = prod_d phi_{m,d,j}(y_td),
// phi_{m,d} a scalar family chosen per dimension (component d of model m)
// with its own parameters per state.  The M-step hands each component the
// same occupancy weights gamma_t(j) and runs that family's own update.
//
// On the device the densities go into the float32 log b table read by the
// recursions (like the other table families), the per-component weighted
// feature sums come from the occupancies (one block per sequence, fixed-order
// float32 partials, then the float64 chunk and model reductions of the
// moment records), and one thread per (model, state, component) applies the
// scalar closed forms / Newton steps of Sec. 4.1-4.3.
//
// Components: Gaussian, Poisson, Gamma, Beta, Student-t, von Mises,
// log-normal, exponential, Rayleigh and chi-squared (the families whose
// M-step reads a fixed set of weighted sums).  Weibull and negative-binomial
// components would need a data pass per Newton step, uniform / Pareto
// components the support extremes; those stay scalar-only.
#pragma once

#include "common.cuh"
#include "ext.cuh"
#include "mstep.cuh"

namespace hmm {

constexpr int INDEP_MAX_D = 32;

__host__ __device__ inline bool indep_component_ok(int f) {
  switch (f) {
    case HMM_GAUSS: case HMM_POISSON: case HMM_GAMMA: case HMM_BETA: case HMM_STUDENT_T: case HMM_VONMISES:
    case HMM_LOGNORMAL: case HMM_EXPONENTIAL: case HMM_RAYLEIGH: case HMM_CHISQ: return true;
    default: return false;
  }
}
__host__ __device__ inline int indep_param_count(int f) {
  switch (f) {
    case HMM_POISSON: case HMM_EXPONENTIAL: case HMM_RAYLEIGH: case HMM_CHISQ: return 1;
    case HMM_STUDENT_T: return 3;
    default: return 2;
  }
}
// weighted sums per component (after the state's shared weight W):
//   GAUSS  S(y-c), S(y-c)^2        POISSON, EXPONENTIAL  Sy
//   GAMMA  Sy, S log y, Sy^2       BETA  Sy, Sy^2, S log y, S log(1-y)
//   STUDENT_T  Su, Su(y-c), Su(y-c)^2, S(log u - u)   (u of Eq. 14)
//   VONMISES  S cos y, S sin y     LOGNORMAL  S(log y - c), S(log y - c)^2
//   RAYLEIGH  Sy^2                 CHISQ  S log y
// with S = sum_t gamma_t(j) and c the component's current float32 shift
// (its mean: Gaussian, Student-t, log-normal of log y).
__host__ __device__ inline int indep_stat_count(int f) {
  switch (f) {
    case HMM_POISSON: case HMM_EXPONENTIAL: case HMM_RAYLEIGH: case HMM_CHISQ: return 1;
    case HMM_GAMMA: return 3;
    case HMM_BETA: case HMM_STUDENT_T: return 4;
    default: return 2;
  }
}
__host__ __device__ inline bool indep_shifted(int f) {
  return f == HMM_GAUSS || f == HMM_STUDENT_T || f == HMM_LOGNORMAL;
}

// Offsets of component d inside a state's parameters and statistics.
struct IndepOff {
  int p, s;
};
__device__ inline IndepOff indep_off(const int* __restrict__ comp, int d) {
  IndepOff o{0, 1};   // statistics start after the shared weight
  for (int e = 0; e < d; ++e) {
    o.p += indep_param_count(comp[e]);
    o.s += indep_stat_count(comp[e]);
  }
  return o;
}

// Derived float32 tables of every (model, state, component): the density
// coefficients (log2 units, as the scalar families) and the shift.
__global__ void indep_derive_kernel(const int* __restrict__ icomp, const double* __restrict__ theta, int M, int NP,
                                    int N, int P, int D, float* __restrict__ icoef, float* __restrict__ ishift) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP * D) return;
  const int d = idx % D, k = (idx / D) % NP, m = idx / (D * NP);
  float* c = icoef + (size_t)idx * KC;
  if (k >= N) {
    for (int z = 0; z < KC; ++z) c[z] = 0.f;
    ishift[idx] = 0.f;
    return;
  }
  const int* comp = icomp + (size_t)m * D;
  const int f = comp[d];
  const double* th = theta + ((size_t)m * NP + k) * P + indep_off(comp, d).p;
  derive_coef(f, th, c, nullptr);
  ishift[idx] = indep_shifted(f) ? (float)th[0] : 0.f;
}

// log b table [total_T][N] (natural log): blocks (sequence, slab of EMIS_SLAB
// rows); a fixed (row, state) slot per thread, the components summed in
// log2 units.
__global__ void indep_emission_kernel(const int* __restrict__ icomp, const float* __restrict__ icoef, int NP, int N,
                                      int D, const float* __restrict__ lfact2, const float* __restrict__ y,
                                      const int64_t* __restrict__ offsets, const int32_t* __restrict__ model_id,
                                      float* __restrict__ logb) {
  const int s = blockIdx.x;
  const int64_t b = offsets[s] + (int64_t)blockIdx.y * EMIS_SLAB;
  const int64_t e = min(offsets[s + 1], b + (int64_t)EMIS_SLAB);
  if (b >= e) return;
  const int m = model_id[s];
  const int* comp = icomp + (size_t)m * D;
  const int rpp = N <= (int)blockDim.x ? blockDim.x / N : 1;
  for (int slot = threadIdx.x; slot < rpp * N; slot += blockDim.x) {
    const int rr = slot / N, k = slot % N;
    const float* cs = icoef + ((size_t)m * NP + k) * D * KC;
    for (int64_t t = b + rr; t < e; t += rpp) {
      float l2 = 0.f;
      for (int d = 0; d < D; ++d) {
        const int f = comp[d];
        const Feat ft = feat_of(f, y[t * D + d], lfact2);
        l2 += ft.ok ? emis_log2(f, ft, cs + d * KC, nullptr) : -INFINITY;
      }
      logb[t * N + k] = l2 * kLn2f;
    }
  }
}

// Weighted feature z (>= 1) of component f at observation v (see
// indep_stat_count); st = (mu, sigma2, nu) of a Student-t component.
__device__ __forceinline__ float indep_feature(int f, int z, float v, float c, const float* st) {
  switch (f) {
    case HMM_GAUSS: {
      const float dv = v - c;
      return z == 0 ? dv : dv * dv;
    }
    case HMM_POISSON:
    case HMM_EXPONENTIAL: return v;
    case HMM_GAMMA: return z == 0 ? v : (z == 1 ? logf(v) : v * v);
    case HMM_BETA: return z == 0 ? v : (z == 1 ? v * v : (z == 2 ? logf(v) : log1pf(-v)));
    case HMM_STUDENT_T: {
      const float r = v - st[0];
      const float u = (st[2] + 1.f) / (st[2] + r * r / st[1]);
      const float dv = v - c;
      return z == 0 ? u : (z == 1 ? u * dv : (z == 2 ? u * dv * dv : logf(u) - u));
    }
    case HMM_VONMISES: return z == 0 ? cosf(v) : sinf(v);
    case HMM_LOGNORMAL: {
      const float dv = logf(v) - c;
      return z == 0 ? dv : dv * dv;
    }
    case HMM_RAYLEIGH: return v * v;
    case HMM_CHISQ: return logf(v);
    default: return 0.f;
  }
}

// Per-sequence weighted sums part[s][NP][KS] (slot 0: W = sum gamma; then
// the components' sums in order).  One block per sequence: thread (pair,
// r) owns pair = (state, slot) and the rows r, r + R, ... of the sequence
// (R = blockDim / pairs), two-level float32 sums (64 rows per inner sum);
// the R partials of a pair are added in fixed order, so the result does not
// depend on scheduling.  Rows of zero weight add nothing (they include the
// rows outside some component's support).
__global__ void __launch_bounds__(256) indep_stats_kernel(const int* __restrict__ icomp, const float* __restrict__ ishift,
                                                          const double* __restrict__ theta, int NP, int N, int D, int P,
                                                          int KS, const float* __restrict__ y,
                                                          const float* __restrict__ gamma,
                                                          const int64_t* __restrict__ offsets,
                                                          const int32_t* __restrict__ model_id,
                                                          float* __restrict__ part) {
  __shared__ float red[256];
  const int s = blockIdx.x;
  const int64_t b = offsets[s], e = offsets[s + 1];
  const int m = model_id[s];
  const int* comp = icomp + (size_t)m * D;
  const int pairs = N * KS;
  for (int p0 = 0; p0 < NP * KS; p0 += blockDim.x) {
    const int npair = min(pairs - p0, (int)blockDim.x);          // pairs of this round (may be <= 0)
    const int R = npair > 0 ? max(1, (int)blockDim.x / npair) : 1;
    const int pair = p0 + (npair > 0 ? (int)threadIdx.x % npair : 0);
    const int r = npair > 0 ? (int)threadIdx.x / npair : 0;
    const bool live = npair > 0 && r < R && pair < pairs;
    float acc = 0.f;
    if (live) {
      const int k = pair / KS, zs = pair % KS;
      // which component and which of its sums
      int d = -1, z = 0, f = 0;
      if (zs > 0) {
        int o = 1;
        for (int dd = 0; dd < D; ++dd) {
          const int n = indep_stat_count(comp[dd]);
          if (zs < o + n) {
            d = dd;
            z = zs - o;
            f = comp[dd];
            break;
          }
          o += n;
        }
      }
      float c = 0.f, st[3] = {0.f, 1.f, 1.f};
      if (d >= 0) {
        c = ishift[((size_t)m * NP + k) * D + d];
        if (f == HMM_STUDENT_T) {
          const double* th = theta + ((size_t)m * NP + k) * P + indep_off(comp, d).p;
          st[0] = (float)th[0];
          st[1] = (float)th[1];
          st[2] = (float)th[2];
        }
      }
      if (zs == 0 || d >= 0) {
        float in = 0.f;
        int cnt = 0;
        for (int64_t t = b + r; t < e; t += R) {
          const float g = gamma[t * N + k];
          if (g > 0.f) in = fmaf(g, d < 0 ? 1.f : indep_feature(f, z, y[t * D + d], c, st), in);
          if (++cnt == 64) {
            acc += in;
            in = 0.f;
            cnt = 0;
          }
        }
        acc += in;
      }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int q = threadIdx.x; q < min((int)blockDim.x, NP * KS - p0); q += blockDim.x) {
      const int pq = p0 + q;
      float v = 0.f;
      if (npair > 0 && q < npair)
        for (int rr = 0; rr < R; ++rr) v += red[rr * npair + q];
      part[(size_t)s * NP * KS + pq] = v;
    }
    __syncthreads();
  }
}

// M-step of every (model, state, component) from the reduced sums
// rec[M][NP][KS] (float64): the scalar updates of Sec. 4.1-4.3 with the
// weights of the state (Sec. 4.5), the collapse guard of Sec. 4.4 on the
// state's W, and an undefined update keeping that component.
__global__ void indep_mstep_kernel(const int* __restrict__ icomp, const float* __restrict__ ishift,
                                   double* __restrict__ theta, const double* __restrict__ rec, int M, int NP, int N,
                                   int P, int D, int KS, MStepOpts o) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP * D) return;
  const int d = idx % D, k = (idx / D) % NP, m = idx / (D * NP);
  if (k >= N) return;
  const int* comp = icomp + (size_t)m * D;
  const int f = comp[d];
  const IndepOff off = indep_off(comp, d);
  const double* R = rec + ((size_t)m * NP + k) * KS;
  const double W = R[0];
  if (!(W >= o.collapse_eps)) return;
  const double* S = R + off.s;
  double* th = theta + ((size_t)m * NP + k) * P + off.p;
  const double c = (double)ishift[((size_t)m * NP + k) * D + d];
  double nt[3] = {th[0], indep_param_count(f) > 1 ? th[1] : 0.0, indep_param_count(f) > 2 ? th[2] : 0.0};
  switch (f) {
    case HMM_GAUSS:
    case HMM_LOGNORMAL: {
      const double d1 = S[0] / W;
      nt[0] = c + d1;
      nt[1] = resolved_var(S[1] / W - d1 * d1, S[1] / W);
      break;
    }
    case HMM_POISSON: nt[0] = S[0] / W; break;
    case HMM_EXPONENTIAL: nt[0] = W / S[0]; break;
    case HMM_RAYLEIGH: nt[0] = S[0] / (2.0 * W); break;
    case HMM_CHISQ: nt[0] = 2.0 * ext_inv_digamma(S[0] / W - kLn2, o); break;
    case HMM_GAMMA: {
      const double ybar = S[0] / W, mlog = S[1] / W, var = S[2] / W - ybar * ybar;
      nt[0] = gamma_shape(ybar, var, log(ybar) - mlog, o);
      nt[1] = nt[0] / ybar;
      break;
    }
    case HMM_BETA: {
      const double ybar = S[0] / W, var = S[1] / W - ybar * ybar;
      beta_fit(ybar, var, S[2] / W, S[3] / W, o, &nt[0], &nt[1]);
      break;
    }
    case HMM_STUDENT_T: {   // Eq. 15-19 with u from the current parameters
      const double d1 = S[1] / S[0];
      nt[0] = c + d1;
      nt[1] = resolved_var((S[2] - S[1] * d1) / W, S[2] / W);
      nt[2] = student_nu(W, S[3], th[2], o);
      break;
    }
    case HMM_VONMISES:
      nt[0] = atan2(S[1], S[0]);
      nt[1] = vonmises_kappa(hypot(S[0], S[1]) / W, o);
      break;
    default: return;
  }
  if (!valid_update(f, nt)) return;
  for (int z = 0; z < indep_param_count(f); ++z) th[z] = nt[z];
}

}  // namespace hmm
