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

#include <type_traits>

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
  int* work_counter;         // [1], or [sched.n_seg]
  int* status;
  FamSched sched;
};

template <int NP_, int G_>
struct SmallCfg {
  static constexpr int NP = NP_;
  static constexpr int G = G_;
  static constexpr int R = NP / G;
  static constexpr int CPW = 32 / G;
  static constexpr int SPW = CPW / 2;
  static constexpr int F = NP + NST;
  static constexpr int PD = 8;          // prefetch ring depth (steps)
  static constexpr int FLUSH = 64;      // inner accumulation length (steps)
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
  float acc[C::R * C::F][32];            // outer sums, field-major / lane-minor
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

// Mode bits of the E-step kernels (compile time).
constexpr int MODE_STATS = 1;   // accumulate xi and the family sums
constexpr int MODE_GAMMA = 2;   // write gamma_t(j) rows

__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <class C, int FAM, int MODE>
__device__ void estep_item(WarpSmem<C>& sm, const EStepArgs& a, int item, int lane) {
  constexpr int NP = C::NP, G = C::G, R = C::R, F = C::F;
  constexpr bool STATS = (MODE & MODE_STATS) != 0;
  constexpr bool GAMMA = (MODE & MODE_GAMMA) != 0;
  constexpr int NH = NP / 2;
  constexpr int PD = C::PD;
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
  int fam = FAM;
  if constexpr (FAM == FAM_ANY) fam = fam_rt;

  // ---- model data of this chain: pairs over the summation index i
  float2 Mb[NH][R];   // forward: (a_{i,k}, a_{i+1,k}); backward: (a_{k,i}, a_{k,i+1})
  const float* Am = a.mv.A32 + (size_t)m * NP * NP;
#pragma unroll
  for (int i = 0; i < NH; ++i)
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int k = k0 + q;
      Mb[i][q] = dir == 0 ? make_float2(__ldg(Am + (2 * i) * NP + k), __ldg(Am + (2 * i + 1) * NP + k))
                          : make_float2(__ldg(Am + k * NP + 2 * i), __ldg(Am + k * NP + 2 * i + 1));
    }
  constexpr bool NEED_NB = (FAM == HMM_NEGBIN || FAM == FAM_ANY);
  constexpr bool NEED_C2 = (FAM == HMM_STUDENT_T || FAM == FAM_ANY);
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
    cf2[q][0] = NEED_C2 ? __ldg(c + 4) : 0.f;
    cf2[q][1] = NEED_C2 ? __ldg(c + 5) : 0.f;
    nbt[q] = (NEED_NB && a.mv.nbtab) ? a.mv.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
  }

  // ---- schedule: phase 1 runs n1 steps (forward t = 0..h-1, backward
  // t = T-1..h), phase 2 runs n2 steps (forward t = h..T-1, backward
  // t = h-1..0).  The warp runs the longest phase of its chains; shorter
  // chains are masked.
  const int n1 = T <= 0 ? 0 : (dir == 0 ? h : T - h);
  const int n2 = T <= 0 ? 0 : (dir == 0 ? T - h : h);
  const int dt = dir == 0 ? 1 : -1;
  const int ta = dir == 0 ? 0 : T - 1;       // phase-1 start
  const int tb = dir == 0 ? h : h - 1;       // phase-2 start
  int K1 = h, K2 = h;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    K1 = max(K1, __shfl_xor_sync(0xffffffffu, K1, o));
    K2 = max(K2, __shfl_xor_sync(0xffffffffu, K2, o));
  }

  // ---- accumulators (two-level: registers for <= FLUSH steps, then global)
  float2 xi[R][NH];
  float st[R][NST];
#pragma unroll
  for (int q = 0; q < R; ++q) {
#pragma unroll
    for (int i = 0; i < NH; ++i) xi[q][i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int z = 0; z < NST; ++z) st[q][z] = 0.f;
  }
  long long off = 0;       // running log2 offset of this chain (outer part)
  float offs = 0.f;        // inner part: integer-valued, exact below 2^24
  // Outer level of the two-level sums: per-lane slots in shared memory
  // (conflict free), added every FLUSH steps; written to the per-sequence
  // partials once at the end of the item.
  if constexpr (STATS) {
#pragma unroll
    for (int f = 0; f < R * F; ++f) sm.acc[f][lane] = 0.f;
  }
  auto flush = [&]() {
    off += (long long)offs;
    offs = 0.f;
    if constexpr (STATS) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
#pragma unroll
        for (int i = 0; i < NH; ++i) {
          sm.acc[q * F + 2 * i][lane] += xi[q][i].x;
          sm.acc[q * F + 2 * i + 1][lane] += xi[q][i].y;
          xi[q][i] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int z = 0; z < NST; ++z) {
          sm.acc[q * F + NP + z][lane] += st[q][z];
          st[q][z] = 0.f;
        }
      }
    }
  };

  float v[R], gl[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    v[q] = 0.f;
    gl[q] = 0.f;
  }
  bool started = false;    // the chain has produced its first vector
  // The first step of a chain reads no previous vector, but the xi update
  // multiplies that buffer by a zero weight: clear it, so that stale shared
  // memory (NaN or inf) cannot turn 0 x buffer into NaN (a chain whose first
  // step falls in phase 2, e.g. the forward chain of a length-1 sequence).
#pragma unroll
  for (int q = 0; q < R; ++q) {
    sm.xbuf[0][chain][k0 + q] = 0.f;
    sm.xbuf[1][chain][k0 + q] = 0.f;
  }
  __syncwarp();
  const float* ybase = a.y + base;
  const float* sbase = a.scratch + base * NP + k0;
  float* wbase = a.scratch + base * NP + k0;

  // prefetch of the step kk of the current phase into ring slot `slot`
  auto prefetch = [&](int kk, int n, int t0, bool ph2, int slot) {
    if (kk >= n) return;
    const int t = t0 + dt * kk;
    if constexpr (FAM == FAM_TABLE) {
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (k0 + q < N) cp_async4(&sm.lring[slot][chain][k0 + q], a.logb + (base + t) * N + k0 + q);
    } else {
      if (sub == 0) cp_async4(&sm.yring[slot][chain], ybase + t);
    }
    if (ph2) {
      const float* src = sbase + (int64_t)t * NP;
      float* dst = &sm.oring[slot][chain][k0];
      if constexpr (R % 4 == 0) {
#pragma unroll
        for (int q = 0; q < R; q += 4) cp_async16(dst + q, src + q);
      } else if constexpr (R == 2) {
        cp_async8(dst, src);
      } else {
        cp_async4(dst, src);
      }
    }
  };

  // emission of the step whose data sit in ring slot `sl` -> lbn / ftn
  float lbn[R];
  Feat ftn;
  auto emission = [&](int sl) {
    if constexpr (FAM == FAM_TABLE) {
      ftn.y = 0.f;
      ftn.a = 0.f;
      ftn.b = 0.f;
      ftn.ok = true;
#pragma unroll
      for (int q = 0; q < R; ++q)
        lbn[q] = (k0 + q < N) ? sm.lring[sl][chain][k0 + q] * kLog2ef : -INFINITY;
    } else {
      ftn = feat_of(fam, sm.yring[sl][chain], a.mv.lfact2);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        // padding states carry a -inf constant (see derive_row)
        const float e = emis_log2(fam, ftn, cf[q], nbt[q]);
        lbn[q] = ftn.ok ? e : -INFINITY;
      }
    }
  };

  // one recursion step of phase PH2 (false: phase 1) at warp iteration k
  auto step = [&](auto ph2_tag, int k, int n, int t0, int& slot, int& pslot, int xb) {
    constexpr bool PH2 = decltype(ph2_tag)::value;
    const bool act = k < n;
    const int t = t0 + dt * k;
    if (act && started) {
#pragma unroll
      for (int q = 0; q < R; ++q) sm.xbuf[xb][chain][k0 + q] = v[q];
    }
    cp_wait<PD - 3>();      // this step's and the next step's data are in
    __syncwarp();
    prefetch(k + PD - 1, n, t0, PH2, pslot);
    cp_commit();
    pslot = (pslot == PD - 1) ? 0 : pslot + 1;

    // emission log2 b_k(y_t) of the owned states: computed one step ahead
    // (it does not depend on the recursion, so it overlaps the previous step)
    float lb[R];
#pragma unroll
    for (int q = 0; q < R; ++q) lb[q] = lbn[q];
    const Feat ft = ftn;
    emission((slot == PD - 1) ? 0 : slot + 1);
    // mat-vec s = M^T v_prev (or the initial vector), packed FP32x2 FMAs
    const bool first = !started;
    float2 vin[NH];
    load_row<NP>(&sm.xbuf[xb][chain][0], reinterpret_cast<float*>(vin));
    float s[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      float2 e0 = make_float2(0.f, 0.f), e1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NH; i += 2) {
        e0 = __ffma2_rn(vin[i], Mb[i][q], e0);
        if (i + 1 < NH) e1 = __ffma2_rn(vin[i + 1], Mb[i + 1][q], e1);
      }
      s[q] = first ? init[q] : (e0.x + e0.y) + (e1.x + e1.y);
    }

    if constexpr (PH2) {
      float o[R];
#pragma unroll
      for (int q = 0; q < R; ++q) o[q] = sm.oring[slot][chain][k0 + q];
      float zl = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) zl = fmaf(s[q], o[q], zl);
      const float Z = group_sum<G>(zl);
      const bool bfirst = (dir == 1) && (k == 0);
      if (k == 0) {   // warp-uniform: log P(y) at the backward chain's first phase-2 step
        if (bfirst && sub == 0 && act) {
          const long long of = sm.offf[pair];
          double ll = (Z > 0.f) ? ((double)log2f(Z) + (double)(off + (long long)offs + of)) * kLn2
                                : -INFINITY;
          if (!(Z == Z)) {
            ll = NAN;
            set_status(a.status, ST_NUMERIC);
          }
          if (a.loglik && valid) a.loglik[seq] = ll;
        }
      }
      const float rz = (act && Z > 0.f) ? rcpf(Z) : 0.f;
      float w[R], g[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        w[q] = o[q] * rz;
        g[q] = s[q] * w[q];
        gl[q] = act ? g[q] : gl[q];
      }
      if constexpr (STATS) {
       if (act) {
        // xi between the previous and the current step (not at the
        // backward's first phase-2 step: the forward chain counts that pair)
        const float xs = (first || bfirst) ? 0.f : 1.f;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const float wq = w[q] * xs;
          const float2 w2 = make_float2(wq, wq);
#pragma unroll
          for (int i = 0; i < NH; ++i) xi[q][i] = __ffma2_rn(vin[i], w2, xi[q][i]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
          st[q][0] += g[q];
          if constexpr (FAM != FAM_TABLE) accumulate_stats(fam, ft, cf[q], cf2[q], g[q], st[q]);
        }
       }
      }
      if constexpr (GAMMA) {
        if (act) {
          float* gr = a.gamma + (base + t) * (int64_t)N;
#pragma unroll
          for (int q = 0; q < R; ++q)
            if (k0 + q < N) gr[k0 + q] = g[q];
        }
      }
    }

    // new vector: v = s * 2^(lb - E), E = floor(max_j(lb_j + log2 s_j))
    float tm = -INFINITY;
#pragma unroll
    for (int q = 0; q < R; ++q) tm = fmaxf(tm, lb[q] + lg2a(s[q]));
    tm = group_max<G>(tm);
    const float E = (tm > -INFINITY) ? floorf(tm) : 0.f;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const float nv = s[q] * ex2f(lb[q] - E);
      v[q] = act ? nv : v[q];
    }
    if (act) {
      offs += E;
      started = true;
    }
    if constexpr (!PH2) {
      if (act) {
        float* dst = wbase + (int64_t)t * NP;
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
      }
    }
    slot = (slot == PD - 1) ? 0 : slot + 1;
  };


  // ---- phase 1
  int slot = 0, pslot = PD - 1;
#pragma unroll
  for (int kk = 0; kk < PD - 1; ++kk) {
    prefetch(kk, n1, ta, false, kk);
    cp_commit();
  }
  int xb = 0;
  cp_wait<PD - 2>();
  __syncwarp();
  emission(0);
  for (int k = 0; k < K1; ++k) {
    step(std::false_type{}, k, n1, ta, slot, pslot, xb);
    xb ^= 1;
    if ((k & (C::FLUSH - 1)) == C::FLUSH - 1) flush();
  }
  if (dir == 0 && sub == 0) sm.offf[pair] = off + (long long)offs;
  cp_wait<0>();
  __syncwarp();   // phase-1 rows of both chains are visible from here on

  // ---- phase 2
  slot = 0;
  pslot = PD - 1;
#pragma unroll
  for (int kk = 0; kk < PD - 1; ++kk) {
    prefetch(kk, n2, tb, true, kk);
    cp_commit();
  }
  cp_wait<PD - 2>();
  __syncwarp();
  emission(0);
  for (int k = 0; k < K2; ++k) {
    step(std::true_type{}, k, n2, tb, slot, pslot, xb);
    xb ^= 1;
    if ((k & (C::FLUSH - 1)) == C::FLUSH - 1) flush();
  }
  // gamma_1 (the backward chain's last occupancy) feeds the pi update
  if constexpr (STATS) {
    if (dir == 1 && T > 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) st[q][NST - 1] += gl[q];
    }
  }
  flush();
  if constexpr (STATS) {
    if (valid) {
      float* part = a.partials + ((size_t)seq * 2 + dir) * NP * F + (size_t)k0 * F;
#pragma unroll
      for (int f = 0; f < R * F; ++f) part[f] = sm.acc[f][lane];
    }
  }
  cp_wait<0>();
  __syncwarp();
  if (valid && T == 0 && dir == 1 && sub == 0 && a.loglik) a.loglik[seq] = 0.0;
}

}  // namespace hmm

namespace hmm {

// Persistent launch: warps pull work items (SPW sequences each) from global
// counters (for_each_item); items are laid out in the plan's order.
// FAMK: one emission family for the whole launch, FAM_TABLE for a log b
// table, or FAM_ANY for batches that mix families (each work item then runs
// the loop of its family; items mixing families switch per step).
// Specialised launches keep the register budget of the single-family case low.
template <int NP, int G, int WPB, int MODE, int FAMK>
__global__ void __launch_bounds__(WPB * 32) estep_small_kernel(EStepArgs a) {
  using C = SmallCfg<NP, G>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<C>& sm = reinterpret_cast<WarpSmem<C>*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for_each_item(a.sched, a.work_counter, a.n_items, C::SPW, lane, [&](int item) {
    if constexpr (FAMK != FAM_ANY) {
      estep_item<C, FAMK, MODE>(sm, a, item, lane);
    } else {
      // mixed batch: a work item whose chains share one family runs that
      // family's loop; items straddling two families switch per step
      const int pair = (lane / G) >> 1;
      const int slotseq = item * C::SPW + pair;
      const int fam = slotseq < a.n_seq ? a.mv.family[a.model_id[a.order[slotseq]]] : -2;
      const int fam0 = __shfl_sync(0xffffffffu, fam, 0);
      const bool uniform = __all_sync(0xffffffffu, fam == fam0 || fam == -2);
      switch (uniform ? fam0 : FAM_ANY) {
        case HMM_GAUSS: estep_item<C, HMM_GAUSS, MODE>(sm, a, item, lane); break;
        case HMM_POISSON: estep_item<C, HMM_POISSON, MODE>(sm, a, item, lane); break;
        case HMM_NEGBIN: estep_item<C, HMM_NEGBIN, MODE>(sm, a, item, lane); break;
        case HMM_VONMISES: estep_item<C, HMM_VONMISES, MODE>(sm, a, item, lane); break;
        case HMM_GAMMA: estep_item<C, HMM_GAMMA, MODE>(sm, a, item, lane); break;
        default: estep_item<C, FAM_ANY, MODE>(sm, a, item, lane); break;
      }
    }
  });
}

template <int NP, int G>
constexpr size_t estep_small_smem_per_warp() {
  return sizeof(WarpSmem<SmallCfg<NP, G>>);
}

}  // namespace hmm
