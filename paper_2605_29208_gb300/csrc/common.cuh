// Shared device-side definitions of the hmmgpu library (sm_103a).
//
// Units: inside the kernels every log-quantity is kept in base 2
// (log2 b_j(y), log2 a_ij) so that exponentials are single ex2 operations;
// results leave the library in natural-log units (x ln 2 in float64).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hmmgpu.h"

namespace hmm {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;
constexpr float kLog2ef = 1.44269504088896340736f;
constexpr float kLn2f = 0.69314718055994530942f;

// Emission coefficients per (model, state), float32, log2 units.
constexpr int KC = 8;
// Sufficient-statistic slots per state accumulated by the E-step kernels
// (family sums, slot NST-1 holds gamma_1).
constexpr int NST = 6;
// Negative-binomial log2 table: lgamma(y+r) - lgamma(r) - lgamma(y+1) in
// log2 units for integer y < NB_YMAX, computed in float64 per (model, state).
constexpr int NB_YMAX = 512;
// log2(y!) table for integer y < LF_YMAX (Poisson), float64 -> float32.
constexpr int LF_YMAX = 1024;
// Rows per block of the emission-table kernels (grid: sequence x slab).
constexpr long long EMIS_SLAB = 4096;

// Device status word bits (sticky, read by hmm_ctx_status).
enum : int {
  ST_NUMERIC = 1,      // non-finite value met in a recursion
  ST_TIMEOUT = 2,      // bounded wait expired
  ST_ARG = 4           // inconsistent batch (offsets) seen by a kernel
};

// Read-only view of the device-resident models used by all kernels.
struct ModelView {
  int M;              // models
  int N;              // states (real)
  int NP;             // states padded to the kernel size (>= N)
  int D;              // observation dimension
  const int* family;  // [M]
  const float* A32;   // [M][NP][NP] linear a_ij (padded entries 0)
  const float* AT32;  // [M][NP][NP] transposed (padded N > 32 only)
  const float* logA2; // [M][NP][NP] log2 a_ij (-inf for 0)
  const float* logAe; // [M][NP][NP] ln a_ij as float32 (table-mode Viterbi)
  const float* pi32;  // [M][NP]
  const float* logpi2;// [M][NP]
  const float* logpie;// [M][NP]
  const float* coef;  // [M][NP][KC]
  const float* nbtab; // [M][NP][NB_YMAX] or nullptr
  const float* lfact2;// [LF_YMAX] log2(y!)
};

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcpf(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// floor(log2(x)) of a positive normal float from its exponent bits; for 0
// and denormals it gives -127 (the value is only used to pick a shift).
__device__ __forceinline__ float ilog2f(float x) {
  return (float)(int)((__float_as_uint(x) >> 23) & 0xffu) - 127.0f;
}

// Reads an NP-float row of shared memory (16-byte aligned for NP >= 4).
template <int NP>
__device__ __forceinline__ void load_row(const float* src, float* dst) {
  if constexpr (NP % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 4) {
      const float4 t4 = *reinterpret_cast<const float4*>(src + i);
      dst[i] = t4.x;
      dst[i + 1] = t4.y;
      dst[i + 2] = t4.z;
      dst[i + 3] = t4.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NP; i += 2) {
      const float2 t2 = *reinterpret_cast<const float2*>(src + i);
      dst[i] = t2.x;
      dst[i + 1] = t2.y;
    }
  }
}

template <int W>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o, W));
  return v;
}

template <int W>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, W);
  return v;
}

__device__ __forceinline__ void set_status(int* status, int bit) {
  if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------------------
// Emission evaluation.  Per time step a few "features" of y_t are computed
// once and shared by all states; each state then costs 2-5 FP32 operations.
// ---------------------------------------------------------------------------
struct Feat {
  float y;      // observation
  float a;      // family feature 1 (see feat_of)
  float b;      // family feature 2
  bool ok;      // y inside the family's support
};

__device__ __forceinline__ bool is_count(float y) { return y >= 0.f && floorf(y) == y; }

__device__ __forceinline__ Feat feat_of(int fam, float y, const float* __restrict__ lfact2) {
  Feat f;
  f.y = y;
  f.a = 0.f;
  f.b = 0.f;
  f.ok = true;
  switch (fam) {
    case HMM_GAUSS:
    case HMM_STUDENT_T:
      f.ok = (y == y);
      break;
    case HMM_POISSON:
    case HMM_NEGBIN:
      // log2 y!, evaluated in registers: a table read here would put a
      // dependent global load on the recursion's critical path every step
      f.ok = is_count(y);
      f.a = f.ok ? lgammaf(y + 1.0f) * kLog2ef : 0.f;
      break;
    case HMM_GAMMA:
    case HMM_WEIBULL:
      f.ok = y > 0.f;
      f.a = log2f(y);
      break;
    case HMM_BETA:
      f.ok = (y > 0.f) && (y < 1.f);
      f.a = log2f(y);
      f.b = log2f(1.0f - y);
      break;
    case HMM_VONMISES:
      f.ok = (y == y);
      sincosf(y, &f.b, &f.a);  // a = cos y, b = sin y
      break;
    case HMM_LOGNORMAL:
    case HMM_CHISQ:
      f.ok = y > 0.f;
      f.a = log2f(y);
      break;
    case HMM_EXPONENTIAL:
      f.ok = y >= 0.f;
      break;
    case HMM_RAYLEIGH:
      f.ok = y >= 0.f;
      f.a = log2f(y);          // -inf at y = 0: density 0 there
      break;
    case HMM_UNIFORM:          // the support is per state (emis_log2)
      f.ok = (y == y);
      break;
    case HMM_PARETO:
      f.ok = y > 0.f;
      f.a = log2f(y);
      break;
    default:
      break;
  }
  return f;
}

// log2 b_j(y) of one state from its coefficients c[0..KC) (log2 units).
// For the negative binomial `nbt` points at the state's table.
__device__ __forceinline__ float emis_log2(int fam, const Feat& f, const float* c,
                                           const float* __restrict__ nbt) {
  switch (fam) {
    case HMM_GAUSS: {            // c2 - ((y - mu) * c1)^2
      float z = (f.y - c[0]) * c[1];
      return fmaf(-z, z, c[2]);
    }
    case HMM_POISSON:            // y log2 lam - lam log2e - log2 y!
      return fmaf(f.y, c[0], c[1]) - f.a;
    case HMM_GAMMA:              // (alpha-1) log2 y - beta log2e y + const
      return fmaf(c[0], f.a, fmaf(c[1], f.y, c[2]));
    case HMM_BETA:
      return fmaf(c[0], f.a, fmaf(c[1], f.b, c[2]));
    case HMM_WEIBULL: {          // (k-1) log2 y + const - log2e * 2^(k log2 y - k log2 lam)
      float e = ex2f(fmaf(c[1], f.a, c[2]));
      return fmaf(c[0], f.a, fmaf(-kLog2ef, e, c[3]));
    }
    case HMM_NEGBIN: {           // [lgamma(y+r) - lgamma(r)] log2 e - log2 y! + y log2(1-p) + r log2 p
      (void)nbt;
      const float lg = (lgammaf(f.y + c[2]) - c[3]) * kLog2ef - f.a;
      return lg + fmaf(f.y, c[0], c[1]);
    }
    case HMM_STUDENT_T: {        // const - (nu+1)/2 log2(1 + (y-mu)^2 / (nu sigma2))
      float d = f.y - c[0];
      float q = fmaf(d * c[1], d, 1.0f);
      return fmaf(c[2], log2f(q), c[3]);
    }
    case HMM_VONMISES:           // kappa cos(y - mu) log2e + const
      return fmaf(c[0], f.a, fmaf(c[1], f.b, c[2]));
    case HMM_LOGNORMAL: {        // -log2 y + c2 - ((log2 y - mu log2e) c1)^2
      const float z = (f.a - c[0]) * c[1];
      return fmaf(-z, z, c[2]) - f.a;
    }
    case HMM_EXPONENTIAL:        // log2 lam - lam log2e y
      return fmaf(c[0], f.y, c[1]);
    case HMM_RAYLEIGH:           // log2 y - log2 s2 - log2e y^2 / (2 s2)
      return f.a + fmaf(c[0], f.y * f.y, c[1]);
    case HMM_UNIFORM:            // -log2(b - a) on [c0, c1] (bounds rounded inwards to float)
      return (f.y >= c[0] && f.y <= c[1]) ? c[2] : -INFINITY;
    case HMM_CHISQ:              // (nu/2 - 1) log2 y - log2e y / 2 + const
      return fmaf(c[0], f.a, fmaf(c[1], f.y, c[2]));
    case HMM_PARETO:             // log2 alpha + alpha log2 xm - (alpha + 1) log2 y for y >= xm
      return f.y >= c[2] ? fmaf(c[0], f.a, c[1]) : -INFINITY;
    default:
      return 0.f;
  }
}

// The families of the last group (log-normal .. Pareto): density tables,
// statistics from the occupancies (table_stat_count features per row).
__host__ __device__ inline bool is_ext_family(int fam) { return fam >= HMM_LOGNORMAL && fam <= HMM_PARETO; }
__host__ __device__ inline int ext_stat_count(int fam) {
  switch (fam) {
    case HMM_LOGNORMAL: return 3;   // 1, log y, (log y)^2
    case HMM_UNIFORM: return 1;     // 1 (the support min / max come from their own kernel)
    default: return 2;              // 1, and y (exponential), y^2 (Rayleigh), log y (chi-squared, Pareto)
  }
}

// per-row statistic features: slot 0 is the weight
__device__ __forceinline__ float ext_feature(int fam, int z, float y) {
  if (z == 0) return 1.f;
  const float l = y > 0.f ? logf(y) : 0.f;   // rows outside the support carry gamma = 0
  switch (fam) {
    case HMM_LOGNORMAL: return z == 1 ? l : (z == 2 ? l * l : 0.f);
    case HMM_EXPONENTIAL: return z == 1 ? y : 0.f;
    case HMM_RAYLEIGH: return z == 1 ? y * y : 0.f;
    case HMM_CHISQ:
    case HMM_PARETO: return z == 1 ? l : 0.f;
    default: return 0.f;
  }
}


// ---------------------------------------------------------------------------
// Work distribution of the persistent small-N kernels.  Warps take work items
// from global counters.  For batches that mix emission families the plan
// lays the processing order out as one segment per family (each longest
// first) and gives each segment a share of the SMs proportional to its time
// steps: a warp starts on the segment of its SM and moves to the next
// segment once its own is drained.  An SM then runs one family's loop at a
// time (mixed SMs thrash the instruction cache with every family's unrolled
// step), while each segment still starts with its longest sequences.
// ---------------------------------------------------------------------------
struct FamSched {
  int32_t n_seg = 0;                 // 0: one counter over all items
  const int32_t* seg_seq = nullptr;  // [n_seg + 1] segment boundaries in the order
  const int32_t* seg_sm = nullptr;   // [n_seg + 1] SM boundaries: SM s starts on segment f when seg_sm[f] <= s
};

template <class Run>
__device__ __forceinline__ void for_each_item(const FamSched& fs, int* counters, int n_items, int spw, int lane,
                                              Run&& run) {
  if (fs.n_seg <= 0) {
    for (;;) {
      int item = 0;
      if (lane == 0) item = atomicAdd(counters, 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item >= n_items) return;
      run(item);
    }
  }
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  const int nsm = max(fs.seg_sm[fs.n_seg], 1);
  const int sm = (int)(smid % (uint32_t)nsm);
  int home = 0;
  for (int f = 1; f < fs.n_seg; ++f)
    if (sm >= fs.seg_sm[f]) home = f;
  for (int d = 0; d < fs.n_seg; ++d) {
    const int f = (home + d) % fs.n_seg;
    // item i belongs to the segment of its first sequence
    const int ilo = (fs.seg_seq[f] + spw - 1) / spw;
    const int ihi = min(n_items, (fs.seg_seq[f + 1] + spw - 1) / spw);
    for (;;) {
      int item = 0;
      if (lane == 0) item = ilo + atomicAdd(counters + f, 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item >= ihi) break;
      run(item);
    }
  }
}

}  // namespace hmm
