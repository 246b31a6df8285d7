// Max-plus Viterbi decoding (paper Sec. 3.3, Eq. 3-4) for small state
// counts, one persistent launch over a packed ragged batch.
//
// Each sequence is decoded by two chains of G lanes that meet in the middle
// (h = floor(T/2)); lane l of a chain owns R = NP/G states.
//   forward chain, t = 0..h:     delta_t(j) = max_i [delta_{t-1}(i) + log a_ij]
//                                             + log b_j(y_t),
//                                psi_t(j) = argmax_i       (stored in row t)
//   backward chain, t = T-1..h:  beta_{T-1}(i) = 0,
//                                beta_t(i) = max_j [log a_ij + log b_j(y_{t+1})
//                                                   + beta_{t+1}(j)],
//                                phi_t(i) = argmax_j       (stored in row t+1)
// The best path's score is max_j delta_h(j) + beta_h(j) (the max-plus form of
// P(y) = sum_j alpha_h(j) beta_h(j)); with q_h the lowest j attaining it, the
// forward chain traces q_{t-1} = psi_t(q_t) down to t = 0 and the backward
// chain follows q_{t+1} = phi_t(q_t) up to T-1, each on its own half.  The
// decoded path attains the maximum of Eq. 3 (the same score as one forward
// sweep; on exact ties it may pick another maximiser).  Ties inside a step
// keep the lowest index.
//
// After each step a chain subtracts its maximum m_t (added to a float64
// offset) so the scores stay O(1).  With a float32 log-emission table the
// operations are float32 additions, subtractions and comparisons only, so the
// decoded path is a deterministic function of the float32 inputs.  Pointers
// are bytes [total_T][NP]; the tracebacks stage TBCH rows at a time in shared
// memory and walk them there.
#pragma once

#include "common.cuh"
#include "estep_small.cuh"

namespace hmm {

struct VitArgs {
  const float* y;
  const float* logb;          // [total_T][N] natural log (table mode)
  const int64_t* offsets;
  const int32_t* model_id;
  const int32_t* order;
  int32_t n_seq;
  int32_t n_items;
  ModelView mv;
  uint8_t* psi;               // [total_T][NP] (+16 bytes of slack)
  int32_t* path;              // [total_T]
  double* score;              // [S]
  int* work_counter;          // [1], or [sched.n_seg]
  int* status;
  FamSched sched;
};

template <int NP_, int G_>
struct VitCfg {
  static constexpr int NP = NP_;
  static constexpr int G = G_;
  static constexpr int R = NP / G;
  static constexpr int CPW = 32 / G;         // chains per warp
  static constexpr int SPW = CPW / 2;        // sequences per warp
  static constexpr int PD = 8;
  static constexpr int TBCH = 64;
  static constexpr int TBB = TBCH * NP + 8;   // staged bytes per chain (+ alignment slack)
};

template <class C>
struct alignas(16) VitSmem {
  float xbuf[2][C::CPW][C::NP];
  float yring[C::PD][C::CPW];
  float lring[C::PD][C::CPW][C::NP];
  float fin[C::CPW][C::NP];                  // delta_h / beta_h at the meeting point
  double foff[C::CPW];                       // their offsets
  alignas(16) uint8_t tb[C::CPW][(C::TBB + 15) / 16 * 16];
};

// ring slot kk % PD <- the observation (or log b row) `row` of the sequence
template <class C, int FAM>
__device__ __forceinline__ void vit_prefetch(VitSmem<C>& sm, const VitArgs& a, int kk, int row, int chain, int sub,
                                             int64_t base) {
  const int slot = kk % C::PD;
  if constexpr (FAM == FAM_TABLE) {
#pragma unroll
    for (int q = 0; q < C::R; ++q) {
      const int k = sub * C::R + q;
      if (k < a.mv.N) cp_async4(&sm.lring[slot][chain][k], a.logb + (base + row) * a.mv.N + k);
    }
  } else {
    if (sub == 0) cp_async4(&sm.yring[slot][chain], a.y + base + row);
  }
}

template <class C, int FAM>
__device__ void viterbi_item(VitSmem<C>& sm, const VitArgs& a, int item, int lane) {
  constexpr int NP = C::NP, G = C::G, R = C::R;
  const int chain = lane / G, sub = lane % G, k0 = sub * R;
  const int pair = chain >> 1, dir = chain & 1;
  const int slotseq = item * C::SPW + pair;
  const bool valid = slotseq < a.n_seq;
  const int s = valid ? a.order[slotseq] : 0;
  const int64_t base = valid ? a.offsets[s] : 0;
  const int T = valid ? (int)(a.offsets[s + 1] - base) : 0;
  const int m = valid ? a.model_id[s] : 0;
  const int N = a.mv.N;
  int fam = FAM;
  if constexpr (FAM == FAM_ANY) fam = a.mv.family[m];
  constexpr bool TABLE = (FAM == FAM_TABLE);
  const float* La = (TABLE ? a.mv.logAe : a.mv.logA2) + (size_t)m * NP * NP;

  // meeting point and the steps of this chain: forward t = 0..h (h + 1
  // steps), backward beta_{T-1}..beta_h (T - h steps); step k of the
  // backward chain uses row T - k (its step 0 needs no emission)
  const int h = T / 2;
  const int nsteps = T <= 0 ? 0 : (dir == 0 ? h + 1 : T - h);
  auto row_of = [&](int k) { return dir == 0 ? k : (k == 0 ? T - 1 : T - k); };

  constexpr int NH = NP / 2;
  // pairs over the summation index: forward (log a_{2i,k}, log a_{2i+1,k})
  // for the owned column k; backward (log a_{k,2i}, log a_{k,2i+1}) for the
  // owned row k
  float2 L[NH][R];
#pragma unroll
  for (int i = 0; i < NH; ++i)
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int k = k0 + q;
      L[i][q] = dir == 0 ? make_float2(__ldg(La + (2 * i) * NP + k), __ldg(La + (2 * i + 1) * NP + k))
                         : make_float2(__ldg(La + k * NP + 2 * i), __ldg(La + k * NP + 2 * i + 1));
    }
  float init[R], cf[R][4];
  const float* nbt[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int k = k0 + q;
    init[q] = dir == 0 ? __ldg((TABLE ? a.mv.logpie : a.mv.logpi2) + m * NP + k) : (k < N ? 0.f : -INFINITY);
    const float* c = a.mv.coef + ((size_t)m * NP + k) * KC;
#pragma unroll
    for (int z = 0; z < 4; ++z) cf[q][z] = __ldg(c + z);
    nbt[q] = a.mv.nbtab ? a.mv.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
  }

  int kmax = nsteps;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));

#pragma unroll
  for (int kk = 0; kk < C::PD - 1; ++kk) {
    if (kk < nsteps) vit_prefetch<C, FAM>(sm, a, kk, row_of(kk), chain, sub, base);
    cp_commit();
  }

  float d[R];
#pragma unroll
  for (int q = 0; q < R; ++q) d[q] = -INFINITY;
  double off = 0.0;
  float off_in = 0.f;   // float32 inner sum of the shifts (<= 16 steps)
  // emission of the step in ring slot sl, computed one step ahead of its use
  float lbn[R];
  auto emission = [&](int sl) {
    if constexpr (TABLE) {
#pragma unroll
      for (int q = 0; q < R; ++q) lbn[q] = (k0 + q < N) ? sm.lring[sl][chain][k0 + q] : -INFINITY;
    } else {
      const Feat ft = feat_of(fam, sm.yring[sl][chain], a.mv.lfact2);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const float e = emis_log2(fam, ft, cf[q], nbt[q]);
        lbn[q] = ft.ok ? e : -INFINITY;
      }
    }
  };
  cp_wait<C::PD - 2>();
  __syncwarp();
  emission(0);
  int slot = 0;
  for (int k = 0; k < kmax; ++k) {
    const bool active = k < nsteps;
    float lb[R];
#pragma unroll
    for (int q = 0; q < R; ++q) lb[q] = lbn[q];
    // the vector the step maximises over: forward delta_{t-1}; backward
    // log b(y_{t+1}) + beta_{t+1}
    if (active && k > 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) sm.xbuf[k & 1][chain][k0 + q] = dir == 0 ? d[q] : __fadd_rn(d[q], lb[q]);
    }
    cp_wait<C::PD - 3>();
    __syncwarp();
    if (k + C::PD - 1 < nsteps) vit_prefetch<C, FAM>(sm, a, k + C::PD - 1, row_of(k + C::PD - 1), chain, sub, base);
    cp_commit();
    slot = (slot == C::PD - 1) ? 0 : slot + 1;
    emission(slot);
    uint32_t arg4 = 0;
    float nd[R];
    if (k == 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) nd[q] = dir == 0 ? __fadd_rn(init[q], lb[q]) : init[q];
    } else {
      float2 vin[NH];
      load_row<NP>(&sm.xbuf[k & 1][chain][0], reinterpret_cast<float*>(vin));
      const int prow = dir == 0 ? k : T - k;   // pointer row of this step
#pragma unroll
      for (int q = 0; q < R; ++q) {
        // candidates c_i = v_i + log a (IEEE adds, two per instruction), then
        // a pairwise tournament that keeps the right operand only when it is
        // strictly larger: the winner is the lowest index attaining the
        // maximum, as a strict '>' upward scan gives.
        float cv[NP];
        uint32_t ci[NP];
#pragma unroll
        for (int i = 0; i < NH; ++i) {
          const float2 c2 = __fadd2_rn(vin[i], L[i][q]);
          cv[2 * i] = c2.x;
          cv[2 * i + 1] = c2.y;
          ci[2 * i] = 2 * i;
          ci[2 * i + 1] = 2 * i + 1;
        }
#pragma unroll
        for (int w = 1; w < NP; w <<= 1)
#pragma unroll
          for (int j = 0; j + w < NP; j += 2 * w) {
            const bool take = cv[j + w] > cv[j];
            cv[j] = take ? cv[j + w] : cv[j];
            ci[j] = take ? ci[j + w] : ci[j];
          }
        const float best = cv[0];
        const uint32_t arg = ci[0];
        nd[q] = dir == 0 ? __fadd_rn(best, lb[q]) : best;
        arg4 |= arg << (8 * (q & 3));
        if ((q & 3) == 3 || q == R - 1) {
          if (active) {
            uint8_t* dst = a.psi + (base + prow) * NP + k0 + (q & ~3);
            const int nb = (q & 3) + 1;
            if (nb == 4) *reinterpret_cast<uint32_t*>(dst) = arg4;
            else if (nb == 2) *reinterpret_cast<uint16_t*>(dst) = (uint16_t)arg4;
            else *dst = (uint8_t)arg4;
          }
          arg4 = 0;
        }
      }
    }
    float mloc = -INFINITY;
#pragma unroll
    for (int q = 0; q < R; ++q) mloc = fmaxf(mloc, nd[q]);
    const float mx = group_max<G>(mloc);
    if (active) {
      const bool fin = mx > -INFINITY && mx < INFINITY;
#pragma unroll
      for (int q = 0; q < R; ++q) d[q] = fin ? __fsub_rn(nd[q], mx) : nd[q];
      if (fin) off_in += mx;
      if ((k & 15) == 15) {
        off += (double)off_in;
        off_in = 0.f;
      }
    }
  }
  off += (double)off_in;
  cp_wait<0>();

  // ---- meeting point: c_j = delta_h(j) + beta_h(j); q_h = lowest j attaining the maximum
#pragma unroll
  for (int q = 0; q < R; ++q) sm.fin[chain][k0 + q] = d[q];
  if (sub == 0) sm.foff[chain] = off;
  __syncwarp();
  const int cf0 = chain & ~1;   // the forward chain of this pair
  float bv = -INFINITY;
  int bi = k0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const float c = __fadd_rn(sm.fin[cf0][k0 + q], sm.fin[cf0 + 1][k0 + q]);
    if (c > bv) {
      bv = c;
      bi = k0 + q;
    }
  }
  const float gv = group_max<G>(bv);
  int cand = (bv == gv) ? bi : NP;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o, G));
  const int qh = cand >= NP ? 0 : cand;
  if (valid && dir == 0 && sub == 0) {
    if (T > 0) {
      const double sc = (double)gv + sm.foff[cf0] + sm.foff[cf0 + 1];
      a.score[s] = (gv > -INFINITY) ? (TABLE ? sc : sc * kLn2) : -INFINITY;
    } else {
      a.score[s] = 0.0;
    }
  }

  // ---- tracebacks, TBCH pointer rows at a time staged in shared memory:
  // forward chain rows h, h-1, .., 1 (path[h..0]); backward chain rows
  // h+1, .., T-1 (path[h+1..T-1])
  const int nrows = T <= 0 ? 0 : (dir == 0 ? h : T - 1 - h);   // pointer rows of this chain
  int rmax = nrows;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  const int nch = (rmax + C::TBCH - 1) / C::TBCH;
  int q = qh;
  if (valid && dir == 0 && sub == 0 && T > 0) a.path[base + h] = qh;
  for (int c = 0; c < nch; ++c) {
    // rows [lo, hi] of this chunk that carry pointers
    int lo, hi;
    if (dir == 0) {
      hi = h - c * C::TBCH;
      lo = max(hi - C::TBCH + 1, 1);
    } else {
      lo = h + 1 + c * C::TBCH;
      hi = min(lo + C::TBCH - 1, T - 1);
    }
    __syncwarp();
    if (c * C::TBCH < nrows && lo <= hi) {
      const int64_t b0 = (base + lo) * NP;
      const int64_t b1 = (base + hi + 1) * NP;
      const int64_t a0 = b0 & ~(int64_t)3;
      const int nw = (int)((b1 - a0 + 3) >> 2);
      for (int w = sub; w < nw; w += G) cp_async4(&sm.tb[chain][w * 4], a.psi + a0 + w * 4);
    }
    cp_commit();
    cp_wait<0>();
    __syncwarp();
    if (sub == 0 && valid && c * C::TBCH < nrows && lo <= hi) {
      const int64_t a0 = ((base + lo) * NP) & ~(int64_t)3;
      if (dir == 0) {
        for (int t = hi; t >= lo; --t) {
          q = sm.tb[chain][(base + t) * NP + q - a0];
          a.path[base + t - 1] = q;
        }
      } else {
        for (int t = lo; t <= hi; ++t) {
          q = sm.tb[chain][(base + t) * NP + q - a0];
          a.path[base + t] = q;
        }
      }
    }
  }
  __syncwarp();
}

// FAMK as in the E-step: one family per launch, FAM_TABLE, or FAM_ANY
// (per-item dispatch to the family's loop).
template <int NP, int G, int WPB, int FAMK>
__global__ void __launch_bounds__(WPB * 32) viterbi_small_kernel(VitArgs a) {
  using C = VitCfg<NP, G>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  VitSmem<C>& sm = reinterpret_cast<VitSmem<C>*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for_each_item(a.sched, a.work_counter, a.n_items, C::SPW, lane, [&](int item) {
    if constexpr (FAMK != FAM_ANY) {
      viterbi_item<C, FAMK>(sm, a, item, lane);
    } else {
      const int slotseq = item * C::SPW + (lane / G) / 2;
      const int fam = slotseq < a.n_seq ? a.mv.family[a.model_id[a.order[slotseq]]] : -2;
      const int fam0 = __shfl_sync(0xffffffffu, fam, 0);
      const bool uniform = __all_sync(0xffffffffu, fam == fam0 || fam == -2);
      switch (uniform ? fam0 : FAM_ANY) {
        case HMM_GAUSS: viterbi_item<C, HMM_GAUSS>(sm, a, item, lane); break;
        case HMM_POISSON: viterbi_item<C, HMM_POISSON>(sm, a, item, lane); break;
        case HMM_NEGBIN: viterbi_item<C, HMM_NEGBIN>(sm, a, item, lane); break;
        case HMM_VONMISES: viterbi_item<C, HMM_VONMISES>(sm, a, item, lane); break;
        case HMM_GAMMA: viterbi_item<C, HMM_GAMMA>(sm, a, item, lane); break;
        default: viterbi_item<C, FAM_ANY>(sm, a, item, lane); break;
      }
    }
  });
}

}  // namespace hmm
