// Further scalar families of paper Sec. 4.1 and Sec. 4.2: log-normal,
// exponential, Rayleigh, uniform, chi-squared and Pareto.
//
// Their densities go into the log b table (emission_kernel with the
// coefficients of derive_coef), the recursions read the table, and the
// M-step statistics are formed from the occupancies afterwards:
//   * weighted sums of per-row features (mv_moments_kernel, features of
//     ext_feature): 1, log y, (log y)^2, y or y^2 by family;
//   * for the uniform and Pareto families the min / max of y over the rows
//     of the model's sequences that lie in the state's current support
//     (ext_support_kernel).  That is the row set {t : b_j(y_t) > 0}, which
//     equals {t : gamma_t(j) > 0} when pi and A are strictly positive; the
//     test is a float comparison with the bounds the density uses, so it is
//     exact and order-independent.
// ext_mstep_kernel then applies the closed forms (log-normal: the Gaussian
// M-step on log y; exponential: 1 / ybar; Rayleigh: (2 N_j)^-1 sum gamma
// y^2; uniform: min / max; Pareto: xm = min, alpha = N_j / sum gamma
// log(y / xm)) and, for chi-squared, Newton's method on the score equation
// digamma(nu / 2) = mean_gamma(log y) - log 2 (the Gamma M-step with
// beta = 1/2 fixed, Sec. 4.2).
#pragma once

#include "common.cuh"
#include "mstep.cuh"
#include "special.cuh"

namespace hmm {

// float <-> int keys whose integer order is the float order (atomic min/max)
__device__ __forceinline__ int ext_key(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ext_unkey(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__host__ __device__ inline bool ext_has_support_stats(int fam) { return fam == HMM_UNIFORM || fam == HMM_PARETO; }

// Support extremes mm[M][NP][2]: slot 0 the key of the minimum, slot 1 the
// bitwise complement of the key of the maximum (~ reverses the integer
// order), so that both slots combine with MIN: per block, across blocks and
// across the processes of a data-parallel E-step alike.
// mm <- (key(+inf), ~key(-inf))
__global__ void ext_support_init_kernel(int* __restrict__ mm, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mm[2 * i] = ext_key(INFINITY);
  mm[2 * i + 1] = ~ext_key(-INFINITY);
}

// min / max of y over the rows inside each state's current support; blocks
// (sequence, slab of EMIS_SLAB rows), shared-memory partials per state, one
// global atomic per (block, state).  Dynamic shared memory: 2 N ints.
__global__ void ext_support_kernel(const int* __restrict__ family, const float* __restrict__ coef, int NP, int N,
                                   const float* __restrict__ y, const int64_t* __restrict__ offsets,
                                   const int32_t* __restrict__ model_id, int* __restrict__ mm) {
  extern __shared__ int skey[];   // [N] min keys, then [N] max keys
  const int s = blockIdx.x;
  const int64_t b = offsets[s] + (int64_t)blockIdx.y * EMIS_SLAB;
  const int64_t e = min(offsets[s + 1], b + (int64_t)EMIS_SLAB);
  if (b >= e) return;   // uniform across the block
  const int m = model_id[s];
  const int fam = family[m];
  if (!ext_has_support_stats(fam)) return;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    skey[k] = ext_key(INFINITY);
    skey[N + k] = ext_key(-INFINITY);
  }
  __syncthreads();
  for (int64_t idx = threadIdx.x; idx < (e - b) * N; idx += blockDim.x) {
    const int64_t t = b + idx / N;
    const int k = (int)(idx % N);
    const float v = y[t];
    const float* c = coef + ((size_t)m * NP + k) * KC;
    const bool in = fam == HMM_UNIFORM ? (v >= c[0] && v <= c[1]) : (v >= c[2]);
    if (in) {
      const int key = ext_key(v);
      atomicMin(&skey[k], key);
      if (fam == HMM_UNIFORM) atomicMax(&skey[N + k], key);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    int* g = mm + ((size_t)m * NP + k) * 2;
    if (skey[k] != ext_key(INFINITY)) atomicMin(g, skey[k]);
    if (skey[N + k] != ext_key(-INFINITY)) atomicMin(g + 1, ~skey[N + k]);
  }
}

// digamma(x) = c for x > 0 (digamma increases from -inf to +inf): Newton
// from the starting point of Minka's inverse-digamma approximation, steps
// halved to keep x positive; NaN if it does not converge.
__device__ inline double ext_inv_digamma(double c, const MStepOpts& o) {
  if (!isfinite(c)) return NAN;
  double x = c >= -2.22 ? exp(c) + 0.5 : -1.0 / (c + 0.57721566490153286061);
  for (int it = 0; it < o.newton_maxit; ++it) {
    const double f = digamma_d(x) - c, d = trigamma_d(x);
    const double nw = positive_step(x, f / d);
    if (!(nw > 0.0)) return NAN;
    const bool done = newton_done(x, nw, o.newton_tol);
    x = nw;
    if (done) return x;
  }
  return NAN;
}

// M-step of the families above, one thread per (model, state); R = the
// reduced feature sums [M][NP][KS], mm the support min / max keys.  Runs
// before mstep_kernel, whose derive_row then refreshes the coefficients.
__global__ void ext_mstep_kernel(const int* __restrict__ family, double* __restrict__ theta,
                                 const double* __restrict__ rec, const int* __restrict__ mm, int M, int NP, int N,
                                 int P, int KS, MStepOpts o) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * NP) return;
  const int m = idx / NP, k = idx % NP;
  if (k >= N) return;
  const int fam = family[m];
  if (!is_ext_family(fam)) return;
  const double* R = rec + (size_t)idx * KS;
  const double W = R[0];
  if (!(W >= o.collapse_eps)) return;                 // Sec. 4.4: keep theta_j
  double* th = theta + (size_t)idx * P;
  double nt[2] = {th[0], P > 1 ? th[1] : 0.0};
  switch (fam) {
    case HMM_LOGNORMAL: {                             // Gaussian M-step on log y
      const double mu = R[1] / W, m0 = th[0];
      nt[0] = mu;
      nt[1] = resolved_var(R[2] / W - mu * mu, R[2] / W - 2.0 * m0 * R[1] / W + m0 * m0);
      break;
    }
    case HMM_EXPONENTIAL: nt[0] = W / R[1]; break;    // 1 / ybar
    case HMM_RAYLEIGH: nt[0] = R[1] / (2.0 * W); break;
    case HMM_UNIFORM: {
      const int* g = mm + (size_t)idx * 2;
      nt[0] = (double)ext_unkey(g[0]);
      nt[1] = (double)ext_unkey(~g[1]);
      break;
    }
    case HMM_CHISQ:                                   // digamma(nu/2) = E_w log y - log 2
      nt[0] = 2.0 * ext_inv_digamma(R[1] / W - kLn2, o);
      break;
    case HMM_PARETO: {
      const double xm = (double)ext_unkey(mm[(size_t)idx * 2]);
      nt[0] = xm;
      nt[1] = W / (R[1] - W * log(xm));
      break;
    }
    default: break;
  }
  // an update that is undefined on the state's data keeps theta_j
  if (valid_update(fam, nt)) {
    th[0] = nt[0];
    if (P > 1 && (fam == HMM_LOGNORMAL || fam == HMM_UNIFORM || fam == HMM_PARETO)) th[1] = nt[1];
  }
}

}  // namespace hmm
