// Types shared by the host runtime and the M-step kernels: the device model
// buffers, the layout of the statistic record and the M-step options.
#pragma once

#include "common.cuh"

namespace hmm {

// ---------------------------------------------------------------------------
// Mutable device model (float64 master parameters + derived float32 tables)
// ---------------------------------------------------------------------------
struct ModelBufs {
  int M, N, NP, D, P;       // P: float64 parameters per state (theta stride)
  int* family;              // [M]
  double* pi;               // [M][NP]
  double* A;                // [M][NP][NP]
  double* theta;            // [M][NP][P]
  float* A32;
  float* AT32;              // [M][NP][NP] transposed a_ij (padded N > 32 only, else nullptr)
  float* logA2;
  float* logAe;
  float* pi32;
  float* logpi2;
  float* logpie;
  float* coef;              // [M][NP][KC]
  float* nbtab;             // [M][NP][NB_YMAX] or nullptr
  float* lfact2;            // [LF_YMAX]
};

// Record of one model's sufficient statistics after the E-step reduction
// (float64, internal layout):
//   [0] number of sequences, [1] sum of log-likelihoods,
//   [2, 2+NP) gamma_1 sums,
//   [2+NP, 2+NP+NP*NP) X(i,j) = sum_t v(i) o(j)/Z  (xi without the a_ij factor),
//   then NP x (NST-1) family sums (the E-step's shifted / log2 forms).
__host__ __device__ inline int rec_size(int NP) { return 2 + NP + NP * NP + NP * (NST - 1); }
__host__ __device__ inline int rec_g1(int) { return 2; }
__host__ __device__ inline int rec_xi(int NP) { return 2 + NP; }
__host__ __device__ inline int rec_st(int NP) { return 2 + NP + NP * NP; }

struct MStepOpts {
  double collapse_eps;
  double tikhonov_eps;
  int newton_maxit;
  double newton_tol;
  int nu_mode;
  int update_transitions;
  double prior_A;         // Dirichlet concentration of the rows of A (MAP; <= 1: none)
  double prior_pi;        // Dirichlet concentration of pi (MAP; <= 1: none)
  int hard;               // the xi slots hold transition counts (Viterbi training)
};

// Per-(model, state) Newton state of the families whose M-step re-reads the
// data (Weibull shape, negative-binomial r).
struct DPState {
  double x;        // current iterate (k or r)
  double ybar;     // weighted mean of y (negative binomial)
  double mlog;     // weighted mean of log y (Weibull, the data-pass shift)
  double W;        // sum of occupancies
  int active;      // 1 while Newton runs, 2 when the Weibull scale still needs a pass
  int iters;
};

}  // namespace hmm
