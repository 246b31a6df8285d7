// Special functions used by the M-steps (float64 on the device).
//
// digamma / trigamma: the recurrences psi(x) = psi(x+1) - 1/x and
// psi'(x) = psi'(x+1) + 1/x^2 move the argument to x >= 10, where the
// asymptotic (Stirling-type) expansions in Bernoulli numbers B_2k
//   psi(x)  ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)
//   psi'(x) ~ 1/x + 1/(2x^2) + sum_k B_2k / x^(2k+1)
// (Abramowitz & Stegun 6.3.18 and 6.4.12) are summed to k = 7; the truncation
// error at x = 10 is below 1e-16 relative.
//
// Bessel ratio A(kappa) = I1(kappa)/I0(kappa) (paper Sec. 4.2, Eq. 12) and
// log(2 pi I0(kappa)): CUDA's cyl_bessel_i0/i1 below kappa = 500, above it
// the large-argument expansions of I_nu (A&S 9.7.1):
//   A(k) ~ 1 - 1/(2k) - 1/(8k^2) - 1/(8k^3) - 25/(128k^4)
//   log I0(k) ~ k - log(2 pi k)/2 + log(1 + 1/(8k) + 9/(128k^2) + 225/(3072k^3)).
#pragma once

#include <cuda_runtime.h>

namespace hmm {

// Defined here for x > 0 only (NaN otherwise), so that the shift loops
// below run at most 10 times.
__host__ __device__ inline double digamma_d(double x) {
  if (!(x > 0.0)) return NAN;
  double acc = 0.0;
  while (x < 10.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double r = 1.0 / x, r2 = r * r;
  // B2/2 = 1/12, B4/4 = -1/120, B6/6 = 1/252, B8/8 = -1/240, B10/10 = 1/132,
  // B12/12 = -691/32760, B14/14 = 1/12
  double s = r2 * (1.0 / 12 - r2 * (1.0 / 120 - r2 * (1.0 / 252 - r2 * (1.0 / 240 -
             r2 * (1.0 / 132 - r2 * (691.0 / 32760 - r2 * (1.0 / 12)))))));
  return acc + log(x) - 0.5 * r - s;
}

__host__ __device__ inline double trigamma_d(double x) {
  if (!(x > 0.0)) return NAN;
  double acc = 0.0;
  while (x < 10.0) {
    acc += 1.0 / (x * x);
    x += 1.0;
  }
  const double r = 1.0 / x, r2 = r * r;
  // B2 = 1/6, B4 = -1/30, B6 = 1/42, B8 = -1/30, B10 = 5/66, B12 = -691/2730, B14 = 7/6
  double s = r * r2 * (1.0 / 6 - r2 * (1.0 / 30 - r2 * (1.0 / 42 - r2 * (1.0 / 30 -
             r2 * (5.0 / 66 - r2 * (691.0 / 2730 - r2 * (7.0 / 6)))))));
  return acc + r + 0.5 * r2 + s;
}

// float32 versions for the per-observation Newton data passes
// (shift to x >= 8, expansions to B_8).
__device__ __forceinline__ float digamma_f(float x) {
  if (!(x > 0.f)) return NAN;
  float acc = 0.f;
  while (x < 8.f) {
    acc -= 1.0f / x;
    x += 1.f;
  }
  const float r = 1.0f / x, r2 = r * r;
  const float s = r2 * (1.f / 12 - r2 * (1.f / 120 - r2 * (1.f / 252 - r2 * (1.f / 240))));
  return acc + logf(x) - 0.5f * r - s;
}

__device__ __forceinline__ float trigamma_f(float x) {
  if (!(x > 0.f)) return NAN;
  float acc = 0.f;
  while (x < 8.f) {
    acc += 1.0f / (x * x);
    x += 1.f;
  }
  const float r = 1.0f / x, r2 = r * r;
  const float s = r * r2 * (1.f / 6 - r2 * (1.f / 30 - r2 * (1.f / 42 - r2 * (1.f / 30))));
  return acc + r + 0.5f * r2 + s;
}

__device__ inline double bessel_ratio_d(double k) {
  if (k < 500.0) return cyl_bessel_i1(k) / cyl_bessel_i0(k);
  const double r = 1.0 / k;
  return 1.0 - r * (0.5 + r * (0.125 + r * (0.125 + r * (25.0 / 128))));
}

__device__ inline double log_i0_d(double k) {
  if (k < 500.0) return log(cyl_bessel_i0(k));
  const double r = 1.0 / k;
  return k - 0.5 * log(2.0 * 3.14159265358979323846 * k) +
         log1p(r * (0.125 + r * (9.0 / 128 + r * (225.0 / 3072))));
}

}  // namespace hmm
