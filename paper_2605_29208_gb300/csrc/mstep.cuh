// Cross-sequence reductions, the M-step (paper Sec. 4) and the derived
// single-precision tables used by the inference kernels.
#pragma once

#include "common.cuh"
#include "mstep_types.h"
#include "special.cuh"

namespace hmm {

// Level 1: chunk c of the model-sorted sequence list -> float64 record.
// Each field sums the chunk's sequences in list order (fixed order).
__global__ void reduce_estep_l1(const float* __restrict__ partials, const double* __restrict__ loglik,
                                const int32_t* __restrict__ seq_by_model,
                                const int32_t* __restrict__ chunk_lo, const int32_t* __restrict__ chunk_hi,
                                int NP, double* __restrict__ chunk_rec) {
  const int c = blockIdx.x;
  const int lo = chunk_lo[c], hi = chunk_hi[c];
  const int F = NP + NST;
  const int RS = rec_size(NP);
  double* out = chunk_rec + (size_t)c * RS;
  // the chunk's sequence ids staged once; the sums keep their sequential
  // order (unrolled so that the loads are issued ahead of the additions);
  // gridDim.y blocks share the fields of a chunk
  __shared__ int sidx[64];
  for (int z = threadIdx.x; z < hi - lo && z < 64; z += blockDim.x) sidx[z] = seq_by_model[lo + z];
  __syncthreads();
  auto sq = [&](int q) -> size_t { return q - lo < 64 ? (size_t)sidx[q - lo] : (size_t)seq_by_model[q]; };
  for (int f = blockIdx.y * blockDim.x + threadIdx.x; f < RS; f += gridDim.y * blockDim.x) {
    double acc = 0.0;
    if (f == 0) {
      acc = (double)(hi - lo);
    } else if (f == 1) {
#pragma unroll 8
      for (int q = lo; q < hi; ++q) acc += loglik[sq(q)];
    } else if (f < rec_xi(NP)) {
      const int k = f - rec_g1(NP);
#pragma unroll 8
      for (int q = lo; q < hi; ++q) acc += (double)partials[((sq(q) * 2 + 1) * NP + k) * F + NP + NST - 1];
    } else if (f < rec_st(NP)) {
      const int i = (f - rec_xi(NP)) / NP, j = (f - rec_xi(NP)) % NP;
#pragma unroll 8
      for (int q = lo; q < hi; ++q) {
        const size_t s = sq(q);
        // forward chains accumulate xi with state j as the owned index
        acc += (double)partials[((s * 2 + 0) * NP + j) * F + i];
        acc += (double)partials[((s * 2 + 1) * NP + i) * F + j];
      }
    } else {
      const int k = (f - rec_st(NP)) / (NST - 1), z = (f - rec_st(NP)) % (NST - 1);
#pragma unroll 8
      for (int q = lo; q < hi; ++q) {
        const size_t s = sq(q);
        acc += (double)partials[((s * 2 + 0) * NP + k) * F + NP + z];
        acc += (double)partials[((s * 2 + 1) * NP + k) * F + NP + z];
      }
    }
    out[f] = acc;
  }
}

// Level 2: a model's chunk records in order -> the model's record.
// active (optional): nothing to do when *active == 0 (a Newton data pass
// after every state converged; its update reads nothing)
__global__ void reduce_chunks_l2(const double* __restrict__ chunk_rec,
                                 const int32_t* __restrict__ model_chunk_ptr, int RS,
                                 double* __restrict__ rec, const int* __restrict__ active = nullptr) {
  if (active && *active == 0) return;
  const int m = blockIdx.x;
  const int c0 = model_chunk_ptr[m], c1 = model_chunk_ptr[m + 1];
  for (int f = blockIdx.y * blockDim.x + threadIdx.x; f < RS; f += gridDim.y * blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int c = c0; c < c1; ++c) acc += chunk_rec[(size_t)c * RS + f];
    rec[(size_t)m * RS + f] = acc;
  }
}

// ---------------------------------------------------------------------------
// Derived float32 tables of one state (log2 units for the E-step kernels).
// ---------------------------------------------------------------------------
__device__ inline void derive_coef(int fam, const double* th, float* c, float* nbt) {
#pragma unroll
  for (int z = 0; z < KC; ++z) c[z] = 0.f;
  const double L2E = kLog2e;
  switch (fam) {
    case HMM_GAUSS: {
      const double mu = th[0], s2 = th[1];
      c[0] = (float)mu;
      c[1] = (float)sqrt(L2E / (2.0 * s2));
      c[2] = (float)(-0.5 * log2(2.0 * 3.14159265358979323846 * s2));
      break;
    }
    case HMM_POISSON: {
      const double lam = th[0];
      c[0] = (float)log2(lam);
      c[1] = (float)(-lam * L2E);
      break;
    }
    case HMM_GAMMA: {
      const double a = th[0], b = th[1];
      c[0] = (float)(a - 1.0);
      c[1] = (float)(-b * L2E);
      c[2] = (float)((a * log(b) - lgamma(a)) * L2E);
      break;
    }
    case HMM_BETA: {
      const double a = th[0], b = th[1];
      c[0] = (float)(a - 1.0);
      c[1] = (float)(b - 1.0);
      c[2] = (float)(-(lgamma(a) + lgamma(b) - lgamma(a + b)) * L2E);
      break;
    }
    case HMM_WEIBULL: {
      const double k = th[0], lam = th[1];
      c[0] = (float)(k - 1.0);
      c[1] = (float)k;
      c[2] = (float)(-k * log2(lam));
      c[3] = (float)((log(k) - k * log(lam)) * L2E);
      break;
    }
    case HMM_NEGBIN: {
      const double r = th[0], p = th[1];
      c[0] = (float)log2(1.0 - p);
      c[1] = (float)(r * log2(p));
      c[2] = (float)r;
      c[3] = (float)lgamma(r);
      if (nbt) {
        // T(y) = [lgamma(y+r) - lgamma(r) - lgamma(y+1)] log2 e by the
        // recurrence T(y) = T(y-1) + log((r + y - 1) / y)
        double acc = 0.0;
        nbt[0] = 0.f;
        for (int y = 1; y < NB_YMAX; ++y) {
          acc += log((r + y - 1.0) / (double)y);
          nbt[y] = (float)(acc * L2E);
        }
      }
      break;
    }
    case HMM_STUDENT_T: {
      const double mu = th[0], s2 = th[1], nu = th[2];
      c[0] = (float)mu;
      c[1] = (float)(1.0 / (nu * s2));
      c[2] = (float)(-(nu + 1.0) / 2.0);
      c[3] = (float)((lgamma((nu + 1.0) / 2.0) - lgamma(nu / 2.0) -
                      0.5 * log(nu * 3.14159265358979323846 * s2)) * L2E);
      c[4] = (float)((nu + 1.0) / nu);
      c[5] = (float)log2((nu + 1.0) / nu);
      break;
    }
    case HMM_VONMISES: {
      const double mu = th[0], k = th[1];
      c[0] = (float)(k * cos(mu) * L2E);
      c[1] = (float)(k * sin(mu) * L2E);
      c[2] = (float)(-(log(2.0 * 3.14159265358979323846) + log_i0_d(k)) * L2E);
      break;
    }
    case HMM_LOGNORMAL: {
      const double mu = th[0], s2 = th[1];
      c[0] = (float)(mu * L2E);
      c[1] = (float)sqrt(kLn2 / (2.0 * s2));
      c[2] = (float)(-0.5 * log2(2.0 * 3.14159265358979323846 * s2));
      break;
    }
    case HMM_EXPONENTIAL: {
      const double lam = th[0];
      c[0] = (float)(-lam * L2E);
      c[1] = (float)log2(lam);
      break;
    }
    case HMM_RAYLEIGH: {
      const double s2 = th[0];
      c[0] = (float)(-L2E / (2.0 * s2));
      c[1] = (float)(-log2(s2));
      break;
    }
    case HMM_UNIFORM: {
      // bounds rounded inwards: for a float y, y >= a iff y >= ru(a), y <= b iff y <= rd(b)
      const double a = th[0], b = th[1];
      c[0] = __double2float_ru(a);
      c[1] = __double2float_rd(b);
      c[2] = (float)(-log2(b - a));
      break;
    }
    case HMM_CHISQ: {
      const double h = 0.5 * th[0];
      c[0] = (float)(h - 1.0);
      c[1] = (float)(-0.5 * L2E);
      c[2] = (float)((-h * kLn2 - lgamma(h)) * L2E);
      break;
    }
    case HMM_PARETO: {
      const double xm = th[0], al = th[1];
      c[0] = (float)(-(al + 1.0));
      c[1] = (float)(log2(al) + al * log2(xm));
      c[2] = __double2float_ru(xm);
      break;
    }
    default:
      break;
  }
}

// Coefficient slot that enters log b additively (see emis_log2).
__device__ inline int additive_slot(int fam) {
  switch (fam) {
    case HMM_POISSON:
    case HMM_NEGBIN:
    case HMM_EXPONENTIAL:
    case HMM_RAYLEIGH:
    case HMM_PARETO: return 1;
    case HMM_WEIBULL:
    case HMM_STUDENT_T: return 3;
    default: return 2;
  }
}

// One thread per (model, state row): refresh every derived table of the row.
// the float32 transition tables of entry (m, k, j): linear, transposed, log2, ln
__device__ __forceinline__ void derive_entry(const ModelBufs& mb, int m, int k, int j) {
  const int NP = mb.NP, N = mb.N;
  const size_t row = ((size_t)m * NP + k) * NP;
  const double a = (k < N && j < N) ? mb.A[row + j] : 0.0;
  mb.A32[row + j] = (float)a;
  if (mb.AT32) mb.AT32[((size_t)m * NP + j) * NP + k] = (float)a;
  mb.logA2[row + j] = a > 0.0 ? (float)log2(a) : -INFINITY;
  mb.logAe[row + j] = a > 0.0 ? (float)log(a) : -INFINITY;
}

// tables: also the row's transition tables (float64 logarithms: at large N
// the M-step leaves them to derive_tables_kernel, one thread per entry)
// nbtab: also the negative-binomial count table (511 float64 logarithms; the
// M-step leaves it to nb_table_kernel, one warp per state)
__device__ inline void derive_row(const ModelBufs& mb, int m, int k, bool tables = true, bool nbtab = true) {
  const int NP = mb.NP, N = mb.N;
  if (tables)
    for (int j = 0; j < NP; ++j) derive_entry(mb, m, k, j);
  const double p = k < N ? mb.pi[(size_t)m * NP + k] : 0.0;
  mb.pi32[(size_t)m * NP + k] = (float)p;
  mb.logpi2[(size_t)m * NP + k] = p > 0.0 ? (float)log2(p) : -INFINITY;
  mb.logpie[(size_t)m * NP + k] = p > 0.0 ? (float)log(p) : -INFINITY;
  if (k < N) {
    float* nbt = mb.nbtab ? mb.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
    derive_coef(mb.family[m], mb.theta + ((size_t)m * NP + k) * mb.P,
                mb.coef + ((size_t)m * NP + k) * KC, (nbtab && mb.family[m] == HMM_NEGBIN) ? nbt : nullptr);
  } else {
    // padding state: zero multipliers and a -inf additive constant give
    // log b = -inf for every observation inside the support
    float* c = mb.coef + ((size_t)m * NP + k) * KC;
    for (int z = 0; z < KC; ++z) c[z] = 0.f;
    if (mb.family[m] == HMM_NEGBIN) c[2] = 1.f;   // r = 1 keeps lgamma(y + r) finite
    c[additive_slot(mb.family[m])] = -INFINITY;
  }
}

__global__ void derive_kernel(ModelBufs mb, bool tables = true) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mb.M * mb.NP) return;
  derive_row(mb, idx / mb.NP, idx % mb.NP, tables);
}

__global__ void derive_tables_kernel(ModelBufs mb) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NP = mb.NP;
  if (idx >= (int64_t)mb.M * NP * NP) return;
  derive_entry(mb, (int)(idx / (NP * NP)), (int)(idx / NP % NP), (int)(idx % NP));
}

__global__ void lfact_kernel(float* lfact2) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y < LF_YMAX) lfact2[y] = (float)(lgamma((double)y + 1.0) * kLog2e);
}

// ---------------------------------------------------------------------------
// Newton-Raphson and ECM updates (float64), mirroring Sec. 4.1-4.3.
// ---------------------------------------------------------------------------
__device__ inline bool newton_done(double old, double nw, double tol) {
  return fabs(nw - old) <= tol * fmax(1.0, fabs(old));
}

// Newton step x - step halved until the iterate stays positive, at most 64
// times; NaN when that fails (x itself not positive, or a non-finite step),
// which the M-step then treats as an undefined update.
__device__ inline double positive_step(double x, double step) {
  for (int h = 0; h < 64; ++h) {
    const double nw = x - step;
    if (nw > 0.0 && isfinite(nw)) return nw;
    step *= 0.5;
  }
  return NAN;
}

// Gamma shape by Eq. 7-8 from the MOM seed; c = log ybar - mean log y.
__device__ inline double gamma_shape(double ybar, double var, double c, const MStepOpts& o) {
  // c > 0 unless every weighted observation is equal (no MLE then)
  if (!(c > 0.0) || !(ybar > 0.0)) return NAN;
  // start from the closed-form approximation of the shape MLE given by
  // Minka ("Estimating a Gamma distribution", 2002): within a few per cent,
  // so Newton needs two or three steps
  double a = (3.0 - c + sqrt((c - 3.0) * (c - 3.0) + 24.0 * c)) / (12.0 * c);
  for (int it = 0; it < o.newton_maxit; ++it) {
    const double s = log(a) - digamma_d(a) - c;
    const double ds = 1.0 / a - trigamma_d(a);
    const double nw = positive_step(a, s / ds);
    if (!(nw > 0.0)) return NAN;
    const bool done = newton_done(a, nw, o.newton_tol);
    a = nw;
    if (done) break;
  }
  return a;
}

__device__ inline void beta_fit(double ybar, double var, double m1, double m2, const MStepOpts& o,
                                double* pa, double* pb) {
  const double kk = ybar * (1.0 - ybar) / var - 1.0;
  double a = kk > 0.0 ? ybar * kk : 1.0, b = kk > 0.0 ? (1.0 - ybar) * kk : 1.0;
  for (int it = 0; it < o.newton_maxit; ++it) {
    const double pab = digamma_d(a + b), tab = trigamma_d(a + b);
    const double F0 = digamma_d(a) - pab - m1, F1 = digamma_d(b) - pab - m2;
    const double J00 = trigamma_d(a) - tab, J01 = -tab, J11 = trigamma_d(b) - tab;
    const double det = J00 * J11 - J01 * J01;
    double s0 = (J11 * F0 - J01 * F1) / det, s1 = (J00 * F1 - J01 * F0) / det;
    double na = a - s0, nb = b - s1;
    for (int h = 0; h < 64 && !(na > 0.0 && nb > 0.0); ++h) {
      s0 *= 0.5;
      s1 *= 0.5;
      na = a - s0;
      nb = b - s1;
    }
    if (!(na > 0.0 && nb > 0.0 && isfinite(na) && isfinite(nb))) {
      *pa = NAN;
      *pb = NAN;
      return;
    }
    const bool done = newton_done(a, na, o.newton_tol) && newton_done(b, nb, o.newton_tol);
    a = na;
    b = nb;
    if (done) break;
  }
  *pa = a;
  *pb = b;
}

__device__ inline double vonmises_kappa(double R, const MStepOpts& o) {
  if (R >= 1.0) return 1e6;
  double k = R * (2.0 - R * R) / (1.0 - R * R);
  for (int it = 0; it < o.newton_maxit; ++it) {
    const double A = bessel_ratio_d(k);
    const double dA = 1.0 - A * A - A / k;
    double nw = positive_step(k, (A - R) / dA);
    if (!(nw > 0.0)) return NAN;
    nw = fmin(nw, 1e6);
    const bool done = newton_done(k, nw, o.newton_tol);
    k = nw;
    if (done) break;
  }
  return k;
}

// CM-step 2 of Sec. 4.3 (Eq. 18-19): Newton on nu with C = sum w(log u - u)
// (+ the E[log U] constant in the ECM reading), |d nu| < 1e-6, nu in [0.5, 1e4].
__device__ inline double student_nu(double W, double C, double nu0, const MStepOpts& o) {
  if (o.nu_mode == 0) C += W * (digamma_d(0.5 * (nu0 + 1.0)) - log(0.5 * (nu0 + 1.0)));
  double nu = nu0;
  for (int it = 0; it < o.newton_maxit; ++it) {
    const double g = 0.5 * W * (log(0.5 * nu) + 1.0 - digamma_d(0.5 * nu)) + 0.5 * C;
    const double h = 0.25 * W * (2.0 / nu - trigamma_d(0.5 * nu));
    const double nw = fmin(fmax(nu - g / h, 0.5), 1e4);
    const bool done = fabs(nw - nu) < 1e-6;
    nu = nw;
    if (done) break;
  }
  return nu;
}

// A weighted variance var from float32 sums about the current location
// (msd = the weighted mean square deviation from it): below 1e-6 msd it is
// not resolvable and counts as zero, an undefined update (one observation,
// or all weight on equal values); the oracle applies the same rule.
__host__ __device__ inline double resolved_var(double var, double msd) {
  return var > 1e-6 * msd ? var : 0.0;
}

// Domain check of a closed-form / Newton update (data-pass families are
// checked when their passes finish).
__device__ inline bool valid_update(int fam, const double* th) {
  auto fin = [](double x) { return isfinite(x); };
  switch (fam) {
    case HMM_GAUSS: return fin(th[0]) && fin(th[1]) && th[1] > 0.0;
    case HMM_POISSON: return fin(th[0]) && th[0] > 0.0;
    case HMM_GAMMA: return fin(th[0]) && fin(th[1]) && th[0] > 0.0 && th[1] > 0.0;
    case HMM_BETA: return fin(th[0]) && fin(th[1]) && th[0] > 0.0 && th[1] > 0.0;
    case HMM_STUDENT_T: return fin(th[0]) && fin(th[1]) && fin(th[2]) && th[1] > 0.0 && th[2] > 0.0;
    case HMM_VONMISES: return fin(th[0]) && fin(th[1]) && th[1] >= 0.0;
    case HMM_LOGNORMAL: return fin(th[0]) && fin(th[1]) && th[1] > 0.0;
    case HMM_EXPONENTIAL:
    case HMM_RAYLEIGH:
    case HMM_CHISQ: return fin(th[0]) && th[0] > 0.0;
    case HMM_UNIFORM: return fin(th[0]) && fin(th[1]) && th[0] < th[1];
    case HMM_PARETO: return fin(th[0]) && fin(th[1]) && th[0] > 0.0 && th[1] > 0.0;
    default: return true;
  }
}

// One block per model, one thread per state: emission M-step of state k
// (Sec. 4 with the collapse guard of Sec. 4.4), transition row k and pi_k,
// then the derived tables of row k.  Families whose Newton step needs data
// passes (Weibull, negative binomial) get their seed here and are finished by
// the data-pass kernels.
__global__ void mstep_kernel(ModelBufs mb, const double* __restrict__ rec, MStepOpts o, DPState* dps, bool rows_split) {
  const int m = blockIdx.x, k = threadIdx.x;
  const int NP = mb.NP, N = mb.N;
  if (k >= NP) return;
  const double* R = rec + (size_t)m * rec_size(NP);
  const int fam = mb.family[m];
  if (k < N) {
    double* th = mb.theta + ((size_t)m * NP + k) * mb.P;
    const double* S = R + rec_st(NP) + k * (NST - 1);
    const double W = S[0];
    const float* cf = mb.coef + ((size_t)m * NP + k) * KC;   // current shifts
    if (dps && (fam == HMM_WEIBULL || fam == HMM_NEGBIN)) dps[(size_t)m * NP + k].active = 0;
    double old[4];
    for (int z = 0; z < 4 && z < mb.P; ++z) old[z] = th[z];
    if (W >= o.collapse_eps) {
      switch (fam) {
        case HMM_GAUSS: {
          const double d1 = S[1] / W;
          th[0] = (double)cf[0] + d1;
          th[1] = resolved_var(S[2] / W - d1 * d1, S[2] / W);
          break;
        }
        case HMM_POISSON:
          th[0] = S[1] / W;
          break;
        case HMM_GAMMA: {
          const double ybar = S[1] / W, mlog = S[2] * kLn2 / W;
          const double var = S[3] / W - ybar * ybar;
          const double a = gamma_shape(ybar, var, log(ybar) - mlog, o);
          th[0] = a;
          th[1] = a / ybar;
          break;
        }
        case HMM_BETA: {
          const double ybar = S[1] / W, var = S[2] / W - ybar * ybar;
          beta_fit(ybar, var, S[3] * kLn2 / W, S[4] * kLn2 / W, o, &th[0], &th[1]);
          break;
        }
        case HMM_STUDENT_T: {
          const double Su = S[1], Sud = S[2], Sud2 = S[3];
          const double d1 = Sud / Su;
          const double nu0 = th[2];
          th[0] = (double)cf[0] + d1;                 // Eq. 15
          th[1] = resolved_var((Sud2 - Sud * d1) / W, Sud2 / W);   // Eq. 16 (divides by N_j)
          th[2] = student_nu(W, S[4], nu0, o);        // Eq. 18-19
          break;
        }
        case HMM_WEIBULL: {
          // Eq. 11 reading: seed k0 = pi / (sqrt 6 sd(log y)); Newton runs in the
          // data passes (dp_*), which also finish the scale
          const double mlog = S[1] * kLn2 / W;
          const double vlog = S[2] * kLn2 * kLn2 / W - mlog * mlog;
          DPState& d = dps[(size_t)m * NP + k];
          d.x = 3.14159265358979323846 / (sqrt(6.0) * sqrt(fmax(vlog, 1e-300)));
          d.mlog = mlog;
          d.W = W;
          d.ybar = 0.0;
          d.active = 1;
          d.iters = 0;
          break;
        }
        case HMM_NEGBIN: {
          // profiled score (reading of Sec. 4.2): seed ybar^2 / (var - ybar)
          const double ybar = S[1] / W, var = S[2] / W - ybar * ybar;
          DPState& d = dps[(size_t)m * NP + k];
          d.ybar = ybar;
          d.W = W;
          d.mlog = 0.0;
          d.iters = 0;
          if (var <= ybar) {
            d.x = 1e6;
            d.active = 0;
            th[0] = 1e6;
            th[1] = 1e6 / (1e6 + ybar);
          } else {
            d.x = ybar * ybar / (var - ybar);
            d.active = 1;
          }
          break;
        }
        case HMM_VONMISES: {
          const double C = S[1], Sn = S[2];
          th[0] = atan2(Sn, C);
          th[1] = vonmises_kappa(hypot(C, Sn) / W, o);
          break;
        }
        default:
          break;
      }
      // an update that is undefined on this state's data (non-finite, or
      // outside the family's domain, e.g. a zero weighted variance) keeps
      // theta_j, as the collapse guard of Sec. 4.4 does for a vanishing weight
      if (!valid_update(fam, th))
        for (int z = 0; z < 4 && z < mb.P; ++z) th[z] = old[z];
    }
    if (o.update_transitions) {
      // expected (Baum-Welch: a_ij X_ij) or counted (Viterbi training: X_ij)
      // transitions, plus the Dirichlet pseudo-counts of the MAP reading;
      // from 16 states mstep_rows_kernel updates the rows
      const double cA = o.prior_A > 1.0 ? o.prior_A - 1.0 : 0.0;
      const double cp = o.prior_pi > 1.0 ? o.prior_pi - 1.0 : 0.0;
      if (!rows_split) {
        double* Arow = mb.A + ((size_t)m * NP + k) * NP;
        const double* X = R + rec_xi(NP) + k * NP;
        double den = 0.0;
        for (int j = 0; j < N; ++j) den += (o.hard ? X[j] : Arow[j] * X[j]) + cA;
        if (den >= o.collapse_eps)
          for (int j = 0; j < N; ++j) Arow[j] = ((o.hard ? X[j] : Arow[j] * X[j]) + cA) / den;
      }
      const double ns = R[0];
      if (ns > 0.0) mb.pi[(size_t)m * NP + k] = (R[rec_g1(NP) + k] + cp) / (ns + N * cp);
    }
  }
  __syncthreads();
  derive_row(mb, m, k, !rows_split, false);
}

// T(y) = [lgamma(y + r) - lgamma(r) - lgamma(y + 1)] log2 e for y < NB_YMAX of
// every negative-binomial state: T(y) = sum_{i=1..y} log((r + i - 1) / i),
// lane l of the state's warp adds the terms of y in [16 l, 16 l + 16) and an
// exclusive warp scan (fixed order, float64) gives each lane its start.
static_assert(NB_YMAX == 512, "the count table assumes 16 counts per lane");
__global__ void nb_table_kernel(ModelBufs mb) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= mb.M * mb.NP || !mb.nbtab) return;
  const int m = gw / mb.NP, k = gw % mb.NP;
  if (mb.family[m] != HMM_NEGBIN || k >= mb.N) return;
  const double r = mb.theta[((size_t)m * mb.NP + k) * mb.P];
  double term[16], tot = 0.0;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int yv = 16 * lane + e;
    term[e] = yv == 0 ? 0.0 : log((r + yv - 1.0) / (double)yv);
    tot += term[e];
  }
  double pre = tot;   // inclusive scan of the lane totals
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += u;
  }
  double acc = pre - tot;
  float* nbt = mb.nbtab + ((size_t)m * mb.NP + k) * NB_YMAX;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    acc += term[e];
    nbt[16 * lane + e] = (float)(acc * kLog2e);
  }
}

// Transition row k of model m: expected (Baum-Welch: a_ij X_ij) or counted
// (Viterbi training: X_ij) transitions plus the Dirichlet pseudo-counts of
// the MAP reading, over their sum (128 strided partial sums added by a fixed
// tree).  One block of 128 threads per row; derive_tables_kernel follows.
__global__ void __launch_bounds__(128) mstep_rows_kernel(ModelBufs mb, const double* __restrict__ rec, MStepOpts o) {
  const int NP = mb.NP, N = mb.N;
  const int m = blockIdx.x / NP, k = blockIdx.x % NP, tid = threadIdx.x;
  if (k >= N || !o.update_transitions) return;
  const double* R = rec + (size_t)m * rec_size(NP);
  double* Arow = mb.A + ((size_t)m * NP + k) * NP;
  const double* X = R + rec_xi(NP) + k * NP;
  const double cA = o.prior_A > 1.0 ? o.prior_A - 1.0 : 0.0;
  __shared__ double red[128];
  double part = 0.0;
  for (int j = tid; j < N; j += 128) part += (o.hard ? X[j] : Arow[j] * X[j]) + cA;
  red[tid] = part;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  const double den = red[0];
  if (den >= o.collapse_eps)
    for (int j = tid; j < N; j += 128) Arow[j] = ((o.hard ? X[j] : Arow[j] * X[j]) + cA) / den;
}

// ---------------------------------------------------------------------------
// Data passes for the Newton steps that need the observations again
// (Weibull shape, Eq. 11, and negative-binomial r).
// One warp per sequence, one lane per state, float32 sums over the sequence,
// then the same fixed-order float64 chunk reductions as the E-step.
// Per state three sums:
//   Weibull  S0 = sum g e, S1 = sum g e u, S2 = sum g e u^2 with
//            u = ln y - mlog, e = exp(k u)   (shift mlog cancels in Eq. 11)
//   NegBin   D1 = sum g [psi(y + r) - psi(r)], D2 = sum g [psi'(y + r) - psi'(r)]
// ---------------------------------------------------------------------------
// Lanes cover (time step, state) pairs: lane = tt * NP + k handles state k
// at the steps t = b + tt, b + tt + TPW, ... (TPW = 32 / NP), so a warp reads
// TPW consecutive occupancy rows per iteration; the TPW partial sums of a
// state are combined with shuffles at the end.  Nothing runs once no state
// of any model is active (count in *active_count).
// Negative binomial: the rows with integer y < NB_YMAX enter through the
// weighted histograms of nb_hist_kernel (sum_t gamma_t(j) f(y_t) =
// sum_y h_j(y) f(y), nb_histdot_kernel), so the passes read only the
// sequences that hold larger counts (tail[s] != 0) and add only those rows.
__device__ __forceinline__ void dp_sums_seq(const ModelBufs& mb, const float* __restrict__ y,
                                            const float* __restrict__ gamma, const int64_t* __restrict__ offsets,
                                            const int32_t* __restrict__ model_id, const DPState* __restrict__ dps,
                                            const uint8_t* __restrict__ tail, float* __restrict__ part, int s,
                                            int lane) {
  const int NP = mb.NP, N = mb.N;
  const int TPW = 32 / NP;
  const int tt = lane / NP, k = lane % NP;
  const int m = model_id[s];
  const int fam = mb.family[m];
  float* out = part + (size_t)s * NP * 3;
  const bool dpf = fam == HMM_WEIBULL || (fam == HMM_NEGBIN && tail[s] != 0);
  const DPState* d = dps + (size_t)m * NP;
  const bool mine = dpf && k < N && tt < TPW && d[k].active != 0;
  const bool any = __any_sync(0xffffffffu, mine);
  if (!any) {
    if (lane < NP) {
      out[lane * 3 + 0] = 0.f;
      out[lane * 3 + 1] = 0.f;
      out[lane * 3 + 2] = 0.f;
    }
    return;
  }
  const int64_t b = offsets[s], e = offsets[s + 1];
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  if (mine) {
    const float x = (float)d[k].x;
    float i0 = 0.f, i1 = 0.f, i2 = 0.f;
    int cnt = 0;
    if (fam == HMM_WEIBULL) {
      const float ml = (float)d[k].mlog;
      for (int64_t t = b + tt; t < e; t += TPW) {
        const float g = gamma[t * N + k];
        const float yy = y[t];
        const float u = logf(yy) - ml;
        const float w = (yy > 0.f) ? g * expf(x * u) : 0.f;
        i0 += w;
        i1 = fmaf(w, u, i1);
        i2 = fmaf(w * u, u, i2);
        if (++cnt == 64) {       // two-level sums
          a0 += i0;
          a1 += i1;
          a2 += i2;
          i0 = i1 = i2 = 0.f;
          cnt = 0;
        }
      }
    } else {
      // psi(y + r) - psi(r) and psi'(y + r) - psi'(r) in float32 for the
      // counts >= NB_YMAX (the smaller ones are in the histogram)
      for (int64_t t = b + tt; t < e; t += TPW) {
        const float g = gamma[t * N + k];
        const float yy = y[t];
        const int yi = (int)fminf(yy, 2.0e9f);
        float d1 = 0.f, d2 = 0.f;   // rows below NB_YMAX: in the histogram
        if (yi >= NB_YMAX && g > 0.f) {
          d1 = digamma_f(yy + x) - digamma_f(x);
          d2 = trigamma_f(yy + x) - trigamma_f(x);
        }
        i0 = fmaf(g, d1, i0);
        i1 = fmaf(g, d2, i1);
        if (++cnt == 64) {
          a0 += i0;
          a1 += i1;
          i0 = i1 = 0.f;
          cnt = 0;
        }
      }
    }
    a0 += i0;
    a1 += i1;
    a2 += i2;
  }
  // combine the TPW lanes of each state (fixed xor order: deterministic)
  for (int o = NP; o < 32; o <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane < NP) {
    out[lane * 3 + 0] = a0;
    out[lane * 3 + 1] = a1;
    out[lane * 3 + 2] = a2;
  }
}

__global__ void dp_sums_kernel(ModelBufs mb, const float* __restrict__ y, const float* __restrict__ gamma,
                               const int64_t* __restrict__ offsets, const int32_t* __restrict__ model_id,
                               int n_seq, const DPState* __restrict__ dps, const uint8_t* __restrict__ tail,
                               const int* __restrict__ active_count,
                               float* __restrict__ part) {
  if (*active_count == 0) return;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_seq; s += nwarps)
    dp_sums_seq(mb, y, gamma, offsets, model_id, dps, tail, part, s, lane);
}

// Occupancy-weighted histograms of the integer observations below NB_YMAX
// per negative-binomial state, H[m][NP][NB_YMAX]: fixed-point sums (2^32
// units of gamma, unsigned 64-bit), so that every addition is exact and the
// result does not depend on their order.  One block per row range (about
// 4096 rows) of a chunk of the model-sorted sequence list; a shared-memory
// histogram (dynamic: NP * NB_YMAX * 8 bytes) is flushed once per block with
// global atomics.  tail[s] = 1 marks the sequences holding a count >=
// NB_YMAX.
constexpr double NB_HIST_ONE = 4294967296.0;
__global__ void nb_hist_kernel(ModelBufs mb, const float* __restrict__ y, const float* __restrict__ gamma,
                               const int64_t* __restrict__ offsets, const int32_t* __restrict__ model_id,
                               const int32_t* __restrict__ seq_by_model, const int32_t* __restrict__ chunk_lo,
                               const int32_t* __restrict__ chunk_hi, const int64_t* __restrict__ crow, int split,
                               unsigned long long* __restrict__ H, uint8_t* __restrict__ tail) {
  extern __shared__ unsigned long long hsh[];
  const int c = blockIdx.x;
  const int lo = chunk_lo[c], hi = chunk_hi[c];
  if (lo >= hi) return;
  const int m = model_id[seq_by_model[lo]];
  if (mb.family[m] != HMM_NEGBIN) return;
  const int NP = mb.NP, N = mb.N;
  // block (c, z): rows [z per, (z + 1) per) of the chunk's rows in
  // seq_by_model order (crow[q]: the chunk rows before position q)
  const int slast = seq_by_model[hi - 1];
  const int64_t rows = crow[hi - 1] + (offsets[slast + 1] - offsets[slast]);
  const int64_t per = (rows + split - 1) / split;
  const int64_t zr = (int64_t)blockIdx.y * per;
  const int64_t r0 = zr < rows ? zr : rows, r1 = r0 + per < rows ? r0 + per : rows;
  if (r0 >= r1) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int z = threadIdx.x; z < NP * NB_YMAX; z += blockDim.x) hsh[z] = 0ull;
  __syncthreads();
  // warp w owns the histograms of states w, w + nw, ..: no other warp writes
  // them, and lanes of the warp that hit the same count are merged first, so
  // every update is a plain add of the group's exact fixed-point sum
  for (int k = warp; k < N; k += nw) {
    unsigned long long* hk = hsh + (size_t)k * NB_YMAX;
    for (int q = lo; q < hi; ++q) {
      const int s = seq_by_model[q];
      const int64_t len = offsets[s + 1] - offsets[s], cs = crow[q];
      const int64_t ta = r0 - cs > 0 ? r0 - cs : 0, tb = r1 - cs < len ? r1 - cs : len;
      if (ta >= tb) continue;
      const int64_t b = offsets[s] + ta, e = offsets[s] + tb;
      bool big = false;
      for (int64_t t0 = b; t0 < e; t0 += 32) {
        const int64_t t = t0 + lane;
        int bin = -1;
        unsigned long long v = 0ull;
        if (t < e) {
          const float yy = y[t];
          if (is_count(yy)) {   // density 0 outside the support: no occupancy
            if (yy >= (float)NB_YMAX) {
              big = true;
            } else {
              const float g = gamma[t * N + k];
              if (g > 0.f) {
                bin = (int)yy;
                v = (unsigned long long)llrint((double)g * NB_HIST_ONE);
              }
            }
          }
        }
        const unsigned grp = __match_any_sync(0xffffffffu, bin);
        unsigned long long sum = 0ull;
        for (unsigned mm = grp; mm; mm &= mm - 1) sum += __shfl_sync(grp, v, __ffs(mm) - 1);
        if (bin >= 0 && lane == __ffs(grp) - 1) hk[bin] += sum;
        __syncwarp();
      }
      if (big) tail[s] = 1;
    }
  }
  __syncthreads();
  unsigned long long* Hm = H + (size_t)m * NP * NB_YMAX;
  for (int z = threadIdx.x; z < NP * NB_YMAX; z += blockDim.x)
    if (hsh[z]) atomicAdd(&Hm[z], hsh[z]);
}

// Histogram part of one data pass for every active negative-binomial state:
// sum_y h(y) [psi(y + r) - psi(r)] and sum_y h(y) [psi'(y + r) - psi'(r)]
// over y < NB_YMAX, in float64 from psi(y + r) - psi(r) = sum_{k<y} 1/(r + k)
// and psi'(y + r) - psi'(r) = -sum_{k<y} 1/(r + k)^2 (the recurrences of the
// digamma / trigamma functions), added to the pass's reduced sums.  One warp
// per (model, state): lane l covers y in [16 l, 16 l + 16), an exclusive
// scan of the lanes' increments gives each lane its starting sums; fixed
// order throughout, so the result is deterministic.
static_assert(NB_YMAX == 512, "the histogram dot assumes 16 counts per lane");
__global__ void nb_histdot_kernel(ModelBufs mb, const DPState* __restrict__ dps,
                                  const int* __restrict__ active_count, const unsigned long long* __restrict__ H,
                                  double* __restrict__ dp_rec) {
  if (*active_count == 0) return;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= mb.M * mb.NP) return;
  const int m = w / mb.NP, k = w % mb.NP;
  if (k >= mb.N || mb.family[m] != HMM_NEGBIN || !dps[w].active) return;
  const double r = dps[w].x;
  const int y0 = lane * 16;
  double l1 = 0.0, l2 = 0.0;
  for (int i = 0; i < 16; ++i) {
    const double x = r + (double)(y0 + i);
    l1 += 1.0 / x;
    l2 += 1.0 / (x * x);
  }
  double p1 = l1, p2 = l2;   // inclusive scan over the lanes
  for (int o = 1; o < 32; o <<= 1) {
    const double t1 = __shfl_up_sync(0xffffffffu, p1, o), t2 = __shfl_up_sync(0xffffffffu, p2, o);
    if (lane >= o) {
      p1 += t1;
      p2 += t2;
    }
  }
  double run1 = __shfl_up_sync(0xffffffffu, p1, 1), run2 = __shfl_up_sync(0xffffffffu, p2, 1);
  if (lane == 0) run1 = run2 = 0.0;
  const unsigned long long* h = H + (size_t)w * NB_YMAX;
  double a1 = 0.0, a2 = 0.0;
  for (int i = 0; i < 16; ++i) {
    const double hv = (double)h[y0 + i];
    a1 += hv * run1;
    a2 -= hv * run2;
    const double x = r + (double)(y0 + i);
    run1 += 1.0 / x;
    run2 += 1.0 / (x * x);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    double* R = dp_rec + (size_t)m * mb.NP * 3 + k * 3;
    R[0] += a1 / NB_HIST_ONE;
    R[1] += a2 / NB_HIST_ONE;
  }
}

// plain fixed-order sum of per-sequence records over a chunk of the
// model-sorted sequence list
__global__ void reduce_records_l1(const float* __restrict__ part, int RS, const int32_t* __restrict__ seq_by_model,
                                  const int32_t* __restrict__ chunk_lo, const int32_t* __restrict__ chunk_hi,
                                  double* __restrict__ chunk_rec, const int* __restrict__ active = nullptr) {
  if (active && *active == 0) return;
  const int c = blockIdx.x;
  const int lo = chunk_lo[c], hi = chunk_hi[c];
  for (int f = threadIdx.x; f < RS; f += blockDim.x) {
    double acc = 0.0;
    for (int q = lo; q < hi; ++q) acc += (double)part[(size_t)seq_by_model[q] * RS + f];
    chunk_rec[(size_t)c * RS + f] = acc;
  }
}

// One Newton step per active (model, state); a converged Weibull state asks
// for one more pass to get its scale.  The data-pass sums are float32, so the
// iterate cannot settle below ~1e-7 relative: the stopping tolerance is
// max(newton_tol, 1e-6).  With `final` set every Weibull state still running
// takes its current shape and the scale of the last pass.
__global__ void dp_update_kernel(ModelBufs mb, const double* __restrict__ rec, DPState* dps, MStepOpts o,
                                 int final, const int* __restrict__ active_now, int* __restrict__ active_next) {
  if (*active_now == 0) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mb.M * mb.NP) return;
  const int m = idx / mb.NP, k = idx % mb.NP;
  if (k >= mb.N) return;
  DPState& d = dps[idx];
  if (!d.active) return;
  const int fam = mb.family[m];
  const double* R = rec + (size_t)m * mb.NP * 3 + k * 3;
  double* th = mb.theta + ((size_t)m * mb.NP + k) * mb.P;
  const double tol = fmax(o.newton_tol, 1e-6);
  if (fam == HMM_WEIBULL) {
    const double S0 = R[0], S1 = R[1], S2 = R[2];
    if (d.active == 2 || final) {   // scale from the converged (or last) shape
      const double sc = exp(d.mlog + log(S0 / d.W) / d.x);
      if (d.x > 0.0 && isfinite(d.x) && sc > 0.0 && isfinite(sc)) {
        th[0] = d.x;
        th[1] = sc;
      }
      d.active = 0;
    } else {
      const double kk = d.x;
      const double f = 1.0 / kk - S1 / S0;
      const double df = -1.0 / (kk * kk) - (S2 * S0 - S1 * S1) / (S0 * S0);
      const double nw = positive_step(kk, f / df);
      if (!(nw > 0.0)) {     // undefined on this state's data: keep theta_j
        d.active = 0;
        return;
      }
      d.iters++;
      const bool done = newton_done(kk, nw, tol) || d.iters >= o.newton_maxit;
      d.x = nw;
      if (done) d.active = 2;
    }
  } else if (fam == HMM_NEGBIN) {
    const double r = d.x, W = d.W, ybar = d.ybar;
    const double g = R[0] + W * log(r / (r + ybar));
    const double dg = R[1] + W * (1.0 / r - 1.0 / (r + ybar));
    double nw = positive_step(r, g / dg);
    if (!(nw > 0.0)) {       // undefined on this state's data: keep theta_j
      d.active = 0;
      return;
    }
    nw = fmin(nw, 1e6);
    d.iters++;
    const bool done = newton_done(r, nw, tol) || d.iters >= o.newton_maxit || final;
    d.x = nw;
    th[0] = nw;
    th[1] = nw / (nw + ybar);
    if (done) d.active = 0;
  }
  if (d.active) atomicAdd(active_next, 1);   // still running in the next pass
}

// number of active data-pass states after the seeding M-step
__global__ void dp_count_kernel(const DPState* __restrict__ dps, int n, int* __restrict__ count) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n && dps[idx].active) atomicAdd(count, 1);
}

// refresh the derived tables after the data-pass Newton steps
__global__ void dp_finish_kernel(ModelBufs mb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mb.M * mb.NP) return;
  const int m = idx / mb.NP, k = idx % mb.NP;
  const int fam = mb.family[m];
  if (fam == HMM_WEIBULL || fam == HMM_NEGBIN) derive_row(mb, m, k, true, false);
}

}  // namespace hmm
