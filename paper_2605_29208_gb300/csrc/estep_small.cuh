// Fused E-step for small state counts (padded N <= 64): emission
// log-densities, forward and backward recursions, occupancies gamma and
// pairwise occupancies xi, and the weighted sufficient statistics, in one
// persistent launch over a packed ragged batch.
//
// Method (paper Sec. 3.2): the log-space recursion of Eq. 2,
//   alpha_t(j) = lse_i[alpha_{t-1}(i) + log a_ij] + log b_j(y_t),
// is evaluated in its row-max-shifted exp-space form: every chain keeps
// alpha-hat_t(j) = O_t + log2 v_t(j) with an integer running offset O_t and a
// float32 vector v_t whose largest entry lies in [1, 4).  One step is
//   s_j = sum_i v_{t-1}(i) a_ij                  (mat-vec, FP32 FMAs)
//   E_t = floor(max_j [log2 b_j(y_t) + floor(log2 s_j)])
//   v_t(j) = s_j * 2^(log2 b_j(y_t) - E_t),  O_t = O_{t-1} + E_t,
// which is exactly lse over i of the paper's terms shifted by a per-step
// constant; the shift never loses the scale (no underflow for any T).  The
// backward recursion is the same step with A transposed and the emission
// applied to the new vector (r_t(i) = b_i(y_t) beta_t(i)).
//
// Layout: a "chain" is G lanes of one warp; lane l of a chain owns R = NP/G
// states.  Each warp runs CPW = 32/G chains = SPW = CPW/2 sequences, each as a
// forward chain and a backward chain that meet in the middle:
//   phase 1: forward t = 0..h-1 stores v_t, backward t = T-1..h stores r_t
//            (h = ceil(T/2)), into the row t of a [total_T][NP] scratch;
//   phase 2: forward t = h..T-1 and backward t = h-1..0 continue, reading
//            the partner's stored row at the same t.  With s the mat-vec of
//            the current step and o the partner's row,
//              gamma_t(j) = s_j o_j / Z_t,  Z_t = sum_j s_j o_j,
//            and xi between the previous and the current step is
//            v_prev(i) a_ij o_j / Z_t (forward) or o_i a_ij v_prev(j) / Z_t
//            (backward); the a_ij factor is applied once in the reduction.
//   log P(y) = (log2 Z + O_fwd + O_bwd) ln 2 at the backward chain's first
//   phase-2 step (t = h-1).
// Sufficient statistics and xi sums are accumulated in registers over at most
// FLUSH steps and then added to per-sequence float32 partials in global
// memory (two-level summation); the cross-sequence reduction is a separate,
// fixed-order float64 kernel.
#pragma once

#include "common.cuh"

namespace hmm {

constexpr int FAM_TABLE = 100;   // emissions come from a log b table
constexpr int FAM_ANY = -1;      // family switched per step (mixed warps)

struct EStepArgs {
  const float* y;            // [total_T * D] (scalar families: D = 1)
  const float* logb;         // [total_T][N] natural log, table mode only
  const int64_t* offsets;    // [S+1]
  const int32_t* model_id;   // [S]
  const int32_t* order;      // [S] processing order (family, then length desc)
  int32_t n_seq;
  int32_t n_items;           // work items (SPW sequences each)
  ModelView mv;
  float* scratch;            // [total_T][NP] (may alias gamma when N == NP)
  float* gamma;              // [total_T][N] or nullptr
  float* partials;           // [S][2][NP][NP + NST]
  double* loglik;            // [S] or nullptr
  int* work_counter;
  int* status;
  int want_stats;
};

template <int NP_, int G_>
struct SmallCfg {
  static constexpr int NP = NP_;
  static constexpr int G = G_;
  static constexpr int R = NP / G;
  static constexpr int CPW = 32 / G;
  static constexpr int SPW = CPW / 2;
  static constexpr int F = NP + NST;
  static constexpr int PD = 6;          // prefetch ring depth (iterations)
  static constexpr int GAP = PD - 1;    // idle iterations between the phases
  static constexpr int FLUSH = 64;      // inner accumulation length
  static_assert(NP % G == 0 && G <= 16 && (32 % G) == 0, "bad chain shape");
};

// Shared memory of one warp.
template <class C>
struct alignas(16) WarpSmem {
  float xbuf[2][C::CPW][C::NP];          // exchange of v between a chain's lanes
  float yring[C::PD][C::CPW];            // observations
  float oring[C::PD][C::CPW][C::NP];     // partner rows (phase 2) / logb rows (table)
  float lring[C::PD][C::CPW][C::NP];     // logb rows in table mode
  long long offf[C::SPW];                // forward offsets at the end of phase 1
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

__device__ __forceinline__ bool first_phase2_of_bwd(int k, int h, int gap) { return k == h + gap; }

// Family sums of Sec. 4 for one state with occupancy g (slot 0, the sum of
// g, is added by the caller).  Shifts: Gaussian and Student-t accumulate
// d = y - mu_cur with the float32 mu of the coefficient table.
__device__ __forceinline__ void accumulate_stats(int fam, const Feat& f, const float* c,
                                                 const float* c2, float g, float* st) {
  switch (fam) {
    case HMM_GAUSS: {
      const float d = f.y - c[0], gd = g * d;
      st[1] += gd;
      st[2] = fmaf(gd, d, st[2]);
      break;
    }
    case HMM_POISSON:
      st[1] = fmaf(g, f.y, st[1]);
      break;
    case HMM_GAMMA: {
      const float gy = g * f.y;
      st[1] += gy;
      st[2] = fmaf(g, f.a, st[2]);
      st[3] = fmaf(gy, f.y, st[3]);
      break;
    }
    case HMM_BETA: {
      const float gy = g * f.y;
      st[1] += gy;
      st[2] = fmaf(gy, f.y, st[2]);
      st[3] = fmaf(g, f.a, st[3]);
      st[4] = fmaf(g, f.b, st[4]);
      break;
    }
    case HMM_WEIBULL: {
      const float ga = g * f.a;
      st[1] += ga;
      st[2] = fmaf(ga, f.a, st[2]);
      break;
    }
    case HMM_NEGBIN: {
      const float gy = g * f.y;
      st[1] += gy;
      st[2] = fmaf(gy, f.y, st[2]);
      break;
    }
    case HMM_STUDENT_T: {     // u = (nu+1)/(nu + d^2/sigma2) = c2[0] / q   (Eq. 14)
      const float d = f.y - c[0];
      const float q = fmaf(d * c[1], d, 1.0f);
      const float lq = log2f(q);
      const float u = c2[0] * ex2f(-lq);
      const float lu = (c2[1] - lq) * kLn2f;
      const float gu = g * u;
      st[1] += gu;
      st[2] = fmaf(gu, d, st[2]);
      st[3] = fmaf(gu * d, d, st[3]);
      st[4] = fmaf(g, lu - u, st[4]);
      break;
    }
    case HMM_VONMISES:
      st[1] = fmaf(g, f.a, st[1]);
      st[2] = fmaf(g, f.b, st[2]);
      break;
    default:
      break;
  }
}

// Role of a chain at warp iteration k.
struct Role {
  int t;        // time index, or -1 when idle
  bool phase2;
};

template <class C>
__device__ __forceinline__ Role role_at(int k, int dir, int T, int h) {
  Role r{-1, false};
  if (T <= 0) return r;
  if (dir == 0) {
    if (k < h) r.t = k;
    else if (k >= h + C::GAP && k < T + C::GAP) { r.t = k - C::GAP; r.phase2 = true; }
  } else {
    if (k < T - h) r.t = T - 1 - k;
    else if (k >= h + C::GAP && k < 2 * h + C::GAP) { r.t = 2 * h + C::GAP - 1 - k; r.phase2 = true; }
  }
  return r;
}

// Issue the prefetches that iteration kk needs into ring slot kk % PD.
template <class C, int FAM>
__device__ __forceinline__ void prefetch_iter(WarpSmem<C>& sm, const EStepArgs& a, int kk, int chain,
                                              int sub, int dir, int T, int h, int64_t base) {
  Role r = role_at<C>(kk, dir, T, h);
  if (r.t < 0) return;
  const int slot = kk % C::PD;
  if constexpr (FAM == FAM_TABLE) {
    const int N = a.mv.N;
#pragma unroll
    for (int q = 0; q < C::R; ++q) {
      int k = sub * C::R + q;
      if (k < N) cp_async4(&sm.lring[slot][chain][k], a.logb + (base + r.t) * N + k);
    }
  } else {
    if (sub == 0) cp_async4(&sm.yring[slot][chain], a.y + base + r.t);
  }
  if (r.phase2) {
    const float* src = a.scratch + (base + r.t) * C::NP + sub * C::R;
    float* dst = &sm.oring[slot][chain][sub * C::R];
    if constexpr (C::R % 4 == 0) {
#pragma unroll
      for (int q = 0; q < C::R; q += 4) cp_async16(dst + q, src + q);
    } else if constexpr (C::R == 2) {
      cp_async8(dst, src);
    } else {
      cp_async4(dst, src);
    }
  }
}

template <class C, int FAM>
__device__ void estep_item(WarpSmem<C>& sm, const EStepArgs& a, int item, int lane) {
  constexpr int NP = C::NP, G = C::G, R = C::R, F = C::F;
  const int chain = lane / G, sub = lane % G;
  const int pair = chain >> 1, dir = chain & 1;
  const int slotseq = item * C::SPW + pair;
  const bool valid = slotseq < a.n_seq;
  const int seq = valid ? a.order[slotseq] : 0;
  const int64_t base = valid ? a.offsets[seq] : 0;
  const int T = valid ? (int)(a.offsets[seq + 1] - base) : 0;
  const int h = (T + 1) >> 1;
  const int m = valid ? a.model_id[seq] : 0;
  const int fam_rt = a.mv.family[m];
  const int N = a.mv.N;
  const int k0 = sub * R;

  // ---- model data of this chain
  float Mb[NP][R];   // forward: a_{i, k0+r}; backward: a_{k0+r, i}
  const float* Am = a.mv.A32 + (size_t)m * NP * NP;
#pragma unroll
  for (int i = 0; i < NP; ++i)
#pragma unroll
    for (int q = 0; q < R; ++q)
      Mb[i][q] = dir == 0 ? __ldg(Am + i * NP + k0 + q) : __ldg(Am + (k0 + q) * NP + i);
  float init[R];
  float cf[R][4];
  float cf2[R][2];
  const float* nbt[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int k = k0 + q;
    init[q] = dir == 0 ? __ldg(a.mv.pi32 + m * NP + k) : (k < N ? 1.0f : 0.0f);
    const float* c = a.mv.coef + ((size_t)m * NP + k) * KC;
#pragma unroll
    for (int z = 0; z < 4; ++z) cf[q][z] = __ldg(c + z);
    cf2[q][0] = __ldg(c + 4);
    cf2[q][1] = __ldg(c + 5);
    nbt[q] = a.mv.nbtab ? a.mv.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
  }

  // ---- iteration count of the warp
  int kmax = T > 0 ? 2 * h + C::GAP : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));

  // ---- accumulators
  float xi[R][NP];
  float st[R][NST];
#pragma unroll
  for (int q = 0; q < R; ++q) {
#pragma unroll
    for (int i = 0; i < NP; ++i) xi[q][i] = 0.f;
#pragma unroll
    for (int z = 0; z < NST; ++z) st[q][z] = 0.f;
  }
  float* part = a.partials + ((size_t)(valid ? seq : 0) * 2 + dir) * NP * F + (size_t)k0 * F;
  bool first_flush = true;
  auto flush = [&]() {
    if (valid && a.want_stats) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        float* p = part + q * F;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          p[i] = first_flush ? xi[q][i] : p[i] + xi[q][i];
          xi[q][i] = 0.f;
        }
#pragma unroll
        for (int z = 0; z < NST; ++z) {
          p[NP + z] = first_flush ? st[q][z] : p[NP + z] + st[q][z];
          st[q][z] = 0.f;
        }
      }
    }
    first_flush = false;
  };

  float v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = 0.f;
  long long off = 0;       // running log2 offset of this chain
  bool started = false;    // the chain has produced its first vector

  // ---- prologue prefetch (iterations 0 .. PD-2)
#pragma unroll
  for (int kk = 0; kk < C::PD - 1; ++kk) {
    if (kk < kmax) prefetch_iter<C, FAM>(sm, a, kk, chain, sub, dir, T, h, base);
    cp_commit();
  }

  for (int k = 0; k < kmax; ++k) {
    const Role r = role_at<C>(k, dir, T, h);
    const bool active = r.t >= 0;
    const bool p2 = active && r.phase2;
    const int slot = k % C::PD;

    // publish the previous vector for the mat-vec
    if (active && started) {
#pragma unroll
      for (int q = 0; q < R; ++q) sm.xbuf[k & 1][chain][k0 + q] = v[q];
    }
    cp_wait<C::PD - 2>();
    __syncwarp();
    // refill the slot consumed by iteration k-1 with the data of k+PD-1
    if (k + C::PD - 1 < kmax) prefetch_iter<C, FAM>(sm, a, k + C::PD - 1, chain, sub, dir, T, h, base);
    cp_commit();

    // Every lane runs the arithmetic below (idle chains on stale data) so that
    // the chain-wide shuffles stay convergent; only active chains commit.
    // ---- emission log2 b_k(y_t) for the owned states
    float lb[R];
    int fam = FAM;
    if constexpr (FAM == FAM_ANY) fam = fam_rt;
    Feat ft;
    if constexpr (FAM == FAM_TABLE) {
      ft.y = 0.f;
      ft.a = 0.f;
      ft.b = 0.f;
      ft.ok = true;
#pragma unroll
      for (int q = 0; q < R; ++q)
        lb[q] = (k0 + q < N) ? sm.lring[slot][chain][k0 + q] * kLog2ef : -INFINITY;
    } else {
      ft = feat_of(fam, sm.yring[slot][chain], a.mv.lfact2);
#pragma unroll
      for (int q = 0; q < R; ++q)
        lb[q] = (ft.ok && (k0 + q) < N) ? emis_log2(fam, ft, cf[q], nbt[q]) : -INFINITY;
    }

    // ---- mat-vec s = M^T v_prev (or the initial vector)
    const bool first = !started;
    float s[R];
    float vin[NP];
    load_row<NP>(&sm.xbuf[k & 1][chain][0], vin);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      float e0 = 0.f, e1 = 0.f;
#pragma unroll
      for (int i = 0; i < NP; i += 2) {
        e0 = fmaf(vin[i], Mb[i][q], e0);
        e1 = fmaf(vin[i + 1], Mb[i + 1][q], e1);
      }
      s[q] = first ? init[q] : e0 + e1;
    }

    // ---- phase 2: occupancies, xi and statistics
    float o[R];
#pragma unroll
    for (int q = 0; q < R; ++q) o[q] = sm.oring[slot][chain][k0 + q];
    float zl = 0.f;
#pragma unroll
    for (int q = 0; q < R; ++q) zl = fmaf(s[q], o[q], zl);
    const float Z = group_sum<G>(p2 ? zl : 0.f);
    if (p2) {
      const bool bfirst = (dir == 1) && first_phase2_of_bwd(k, h, C::GAP);
      if (bfirst && sub == 0) {
        // log P(y) = log2 Z + O_bwd + O_fwd  (then x ln 2)
        const long long of = sm.offf[pair];
        double ll = (Z > 0.f) ? ((double)log2f(Z) + (double)(off + of)) * kLn2 : -INFINITY;
        if (!(Z == Z)) {
          ll = NAN;
          set_status(a.status, ST_NUMERIC);
        }
        if (a.loglik && valid) a.loglik[seq] = ll;
      }
      const float rz = (Z > 0.f) ? 1.0f / Z : 0.f;
      float w[R], g[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        w[q] = o[q] * rz;
        g[q] = s[q] * w[q];
      }
      if (a.want_stats) {
        if (!first && !bfirst) {
#pragma unroll
          for (int q = 0; q < R; ++q)
#pragma unroll
            for (int i = 0; i < NP; ++i) xi[q][i] = fmaf(vin[i], w[q], xi[q][i]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const float gq = g[q];
          st[q][0] += gq;
          if constexpr (FAM != FAM_TABLE) accumulate_stats(fam, ft, cf[q], cf2[q], gq, st[q]);
          if (dir == 1 && r.t == 0) st[q][NST - 1] += gq;
        }
      }
      if (a.gamma) {
        float* gr = a.gamma + (base + r.t) * (int64_t)N;
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (k0 + q < N) gr[k0 + q] = g[q];
      }
    }

    // ---- new vector: v = s * 2^(lb - E), E = floor(max(lb + floor(log2 s)))
    float tm = -INFINITY;
#pragma unroll
    for (int q = 0; q < R; ++q) tm = fmaxf(tm, lb[q] + ilog2f(s[q]));
    tm = group_max<G>(tm);
    const float E = (tm > -INFINITY) ? floorf(tm) : 0.f;
    if (active) {
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = s[q] * ex2f(lb[q] - E);
      off += (long long)E;
      started = true;
      if (!r.phase2) {
        // store v_t for the partner's phase 2
        float* dst = a.scratch + (base + r.t) * NP + k0;
        if constexpr (R % 4 == 0) {
#pragma unroll
          for (int q = 0; q < R; q += 4)
            *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        } else if constexpr (R == 2) {
          *reinterpret_cast<float2*>(dst) = make_float2(v[0], v[1]);
        } else {
#pragma unroll
          for (int q = 0; q < R; ++q) dst[q] = v[q];
        }
        if (dir == 0 && r.t == h - 1 && sub == 0) sm.offf[pair] = off;
      }
    }
    if ((k % C::FLUSH) == C::FLUSH - 1) flush();
  }
  flush();
  cp_wait<0>();
  __syncwarp();
  if (valid && T == 0 && dir == 1 && sub == 0 && a.loglik) a.loglik[seq] = 0.0;
}

}  // namespace hmm

namespace hmm {

// Persistent launch: warps pull work items (SPW sequences each) from a
// global counter; items are laid out in the plan's order (family, then
// length descending) so that consecutive items are alike.
template <int NP, int G, int WPB>
__global__ void __launch_bounds__(WPB * 32) estep_small_kernel(EStepArgs a, int table_mode) {
  using C = SmallCfg<NP, G>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<C>& sm = reinterpret_cast<WarpSmem<C>*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.work_counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    if (table_mode) {
      estep_item<C, FAM_TABLE>(sm, a, item, lane);
      continue;
    }
    const int pair = (lane / G) >> 1;
    const int slotseq = item * C::SPW + pair;
    const int fam = slotseq < a.n_seq ? a.mv.family[a.model_id[a.order[slotseq]]] : -2;
    const int fam0 = __shfl_sync(0xffffffffu, fam, 0);
    const bool uniform = __all_sync(0xffffffffu, fam == fam0 || fam == -2);
    switch (uniform ? fam0 : FAM_ANY) {
      case HMM_GAUSS: estep_item<C, HMM_GAUSS>(sm, a, item, lane); break;
      case HMM_POISSON: estep_item<C, HMM_POISSON>(sm, a, item, lane); break;
      case HMM_GAMMA: estep_item<C, HMM_GAMMA>(sm, a, item, lane); break;
      case HMM_BETA: estep_item<C, HMM_BETA>(sm, a, item, lane); break;
      case HMM_WEIBULL: estep_item<C, HMM_WEIBULL>(sm, a, item, lane); break;
      case HMM_NEGBIN: estep_item<C, HMM_NEGBIN>(sm, a, item, lane); break;
      case HMM_STUDENT_T: estep_item<C, HMM_STUDENT_T>(sm, a, item, lane); break;
      case HMM_VONMISES: estep_item<C, HMM_VONMISES>(sm, a, item, lane); break;
      default: estep_item<C, FAM_ANY>(sm, a, item, lane); break;
    }
  }
}

template <int NP, int G>
constexpr size_t estep_small_smem_per_warp() {
  return sizeof(WarpSmem<SmallCfg<NP, G>>);
}

}  // namespace hmm
