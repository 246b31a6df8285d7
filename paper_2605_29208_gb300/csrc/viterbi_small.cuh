// Max-plus Viterbi decoding (paper Sec. 3.3, Eq. 3-4) for small state
// counts, one persistent launch over a packed ragged batch.
//
// A chain of G lanes decodes one sequence; lane l owns R = NP/G states.  Per
// step every owned state j scans its predecessors i upward,
//   c = delta_{t-1}(i) + log a_ij,  keep c if c > best   (lowest i on ties)
//   delta_t(j) = best + log b_j(y_t),  psi_t(j) = argmax,
// then the chain subtracts m_t = max_j delta_t(j) (added to a float64 score)
// so that delta stays O(1).  With a float32 log-emission table the operations
// are float32 additions, subtractions and comparisons only, so the decoded
// path is a deterministic function of the float32 inputs.  Backpointers are
// bytes [total_T][NP]; the traceback stages TBCH rows at a time in shared
// memory and walks them there.
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
  int* work_counter;
  int* status;
};

template <int NP_, int G_>
struct VitCfg {
  static constexpr int NP = NP_;
  static constexpr int G = G_;
  static constexpr int R = NP / G;
  static constexpr int CPW = 32 / G;
  static constexpr int PD = 8;
  static constexpr int TBCH = 64;
  static constexpr int TBB = TBCH * NP + 8;   // staged bytes per chain (+ alignment slack)
};

template <class C>
struct alignas(16) VitSmem {
  float xbuf[2][C::CPW][C::NP];
  float yring[C::PD][C::CPW];
  float lring[C::PD][C::CPW][C::NP];
  alignas(16) uint8_t tb[C::CPW][(C::TBB + 15) / 16 * 16];
};

template <class C, int FAM>
__device__ __forceinline__ void vit_prefetch(VitSmem<C>& sm, const VitArgs& a, int kk, int chain, int sub,
                                             int T, int64_t base) {
  if (kk >= T) return;
  const int slot = kk % C::PD;
  if constexpr (FAM == FAM_TABLE) {
#pragma unroll
    for (int q = 0; q < C::R; ++q) {
      const int k = sub * C::R + q;
      if (k < a.mv.N) cp_async4(&sm.lring[slot][chain][k], a.logb + (base + kk) * a.mv.N + k);
    }
  } else {
    if (sub == 0) cp_async4(&sm.yring[slot][chain], a.y + base + kk);
  }
}

template <class C, int FAM>
__device__ void viterbi_item(VitSmem<C>& sm, const VitArgs& a, int item, int lane) {
  constexpr int NP = C::NP, G = C::G, R = C::R;
  const int chain = lane / G, sub = lane % G, k0 = sub * R;
  const int slotseq = item * C::CPW + chain;
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

  constexpr int NH = NP / 2;
  float2 L[NH][R];   // (log a_{2h,k}, log a_{2h+1,k}) for the owned states k
#pragma unroll
  for (int i = 0; i < NH; ++i)
#pragma unroll
    for (int q = 0; q < R; ++q)
      L[i][q] = make_float2(__ldg(La + (2 * i) * NP + k0 + q), __ldg(La + (2 * i + 1) * NP + k0 + q));
  float init[R], cf[R][4];
  const float* nbt[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int k = k0 + q;
    init[q] = __ldg((TABLE ? a.mv.logpie : a.mv.logpi2) + m * NP + k);
    const float* c = a.mv.coef + ((size_t)m * NP + k) * KC;
#pragma unroll
    for (int z = 0; z < 4; ++z) cf[q][z] = __ldg(c + z);
    nbt[q] = a.mv.nbtab ? a.mv.nbtab + ((size_t)m * NP + k) * NB_YMAX : nullptr;
  }

  int kmax = T;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));

#pragma unroll
  for (int kk = 0; kk < C::PD - 1; ++kk) {
    if (kk < kmax) vit_prefetch<C, FAM>(sm, a, kk, chain, sub, T, base);
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
    const bool active = k < T;
    if (active && k > 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) sm.xbuf[k & 1][chain][k0 + q] = d[q];
    }
    cp_wait<C::PD - 3>();
    __syncwarp();
    if (k + C::PD - 1 < kmax) vit_prefetch<C, FAM>(sm, a, k + C::PD - 1, chain, sub, T, base);
    cp_commit();

    float lb[R];
#pragma unroll
    for (int q = 0; q < R; ++q) lb[q] = lbn[q];
    slot = (slot == C::PD - 1) ? 0 : slot + 1;
    emission(slot);
    uint32_t arg4 = 0;
    float nd[R];
    if (k == 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) nd[q] = __fadd_rn(init[q], lb[q]);
    } else {
      float2 vin[NH];
      load_row<NP>(&sm.xbuf[k & 1][chain][0], reinterpret_cast<float*>(vin));
#pragma unroll
      for (int q = 0; q < R; ++q) {
        // candidates c_i = delta_{t-1}(i) + log a_iq (IEEE adds, two per
        // instruction), then a pairwise tournament that keeps the right
        // operand only when it is strictly larger: the winner is the lowest
        // index attaining the maximum, as a strict '>' upward scan gives.
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
        nd[q] = __fadd_rn(best, lb[q]);
        arg4 |= arg << (8 * (q & 3));
        if ((q & 3) == 3 || q == R - 1) {
          if (active) {
            uint8_t* dst = a.psi + (base + k) * NP + k0 + (q & ~3);
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

  // final state: lowest j attaining the maximum of delta_T
  float bv = -INFINITY;
  int bi = k0;
#pragma unroll
  for (int q = 0; q < R; ++q)
    if (d[q] > bv) {
      bv = d[q];
      bi = k0 + q;
    }
  const float gv = group_max<G>(bv);
  int cand = (bv == gv) ? bi : NP;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o, G));
  int q = cand >= NP ? 0 : cand;
  if (valid && sub == 0 && T > 0) {
    const double sc = (double)gv + off;
    a.score[s] = (gv > -INFINITY) ? (TABLE ? sc : sc * kLn2) : -INFINITY;
  }
  if (valid && sub == 0 && T == 0) a.score[s] = 0.0;

  // ---- traceback, TBCH rows at a time staged in shared memory
  const int nch = (kmax + C::TBCH - 1) / C::TBCH;
  for (int c = 0; c < nch; ++c) {
    const int hi = T - 1 - c * C::TBCH;           // highest row of this chunk
    const int lo = max(hi - C::TBCH + 1, 0);
    __syncwarp();
    if (hi >= 1) {
      const int64_t b0 = (base + max(lo, 1)) * NP;  // rows < 1 carry no pointers
      const int64_t b1 = (base + hi + 1) * NP;
      const int64_t a0 = b0 & ~(int64_t)3;
      const int nw = (int)((b1 - a0 + 3) >> 2);
      for (int w = sub; w < nw; w += G) cp_async4(&sm.tb[chain][w * 4], a.psi + a0 + w * 4);
      cp_commit();
      cp_wait<0>();
    }
    __syncwarp();
    if (sub == 0 && valid && hi >= 0) {
      const int64_t a0 = ((base + max(lo, 1)) * NP) & ~(int64_t)3;
      for (int t = hi; t >= lo; --t) {
        a.path[base + t] = q;
        if (t >= 1) q = sm.tb[chain][(base + t) * NP + q - a0];
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
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.work_counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    if constexpr (FAMK != FAM_ANY) {
      viterbi_item<C, FAMK>(sm, a, item, lane);
    } else {
      const int slotseq = item * C::CPW + lane / G;
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
  }
}

}  // namespace hmm
