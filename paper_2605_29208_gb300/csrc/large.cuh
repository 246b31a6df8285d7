// Large-N inference path: padded state counts 64 ... 1024, float32 CUDA
// cores.  Emissions come from a float32 log b table; the transition matrix
// (1 KB ... 4 MB per model) no longer fits a warp's registers, so a block of
// 256 threads runs a group of LG_SB sequences of one model in lock step and
// reads A once per step for all of them (from shared memory up to N = 128,
// else from L2).
//
// Forward (Eq. 1-2) and backward (Sec. 3.2) run in the same launch (grid.y
// = direction) with the shifted exp-space form of the small-N kernels:
//   forward   v_t = 2^(log2 b_t + log2(A^T v_{t-1}) - E_t),  alpha_t = v_t 2^Oa_t
//   backward  bt_t = A z_{t+1} (stored),  z_t = 2^(log2 b_t + log2 bt_t - E_t),
//             beta_t = bt_t 2^Ob_t  with Ob_t the offset of z_{t+1}
// E_t = floor(max_j(...)) per sequence and step, offsets kept in float64.
// With Z_t = sum_j v_t(j) bt_t(j):
//   gamma_t(j) = v_t(j) bt_t(j) / Z_t,   log L = log2 Z_t + Oa_t + Ob_t (any t)
//   xi_t(i,j) / a_ij = v_t(i) z_{t+1}(j) / Z_t.
#pragma once

#include "common.cuh"
#include "estep_small.cuh"

namespace hmm {

constexpr int LG_SB = 8;     // sequences per group
constexpr int LG_NT = 256;   // threads per block
constexpr int LG_TB = 32;    // Viterbi traceback rows staged per chunk

template <int NP>
struct LgShape {
  static constexpr int CG = NP < LG_NT ? NP : LG_NT;   // column groups (threads per sequence set)
  static constexpr int JC = NP / CG;                    // columns per thread
  static constexpr int TS = LG_NT / CG;                 // sequence sets
  static constexpr int SBT = LG_SB / TS;                // sequences per thread
  static constexpr int WPS = CG / 32;                   // warps per sequence set
  static constexpr bool A_SMEM = NP <= 128;             // A staged in shared memory
  static constexpr size_t smem_bytes() {
    return (size_t)(2 * LG_SB * NP + (LG_NT / 32) * LG_SB) * 4 + (A_SMEM ? (size_t)NP * NP * 4 : 0);
  }
};

struct LargeArgs {
  const float* logb;           // [total_T][N] natural log
  const int64_t* offsets;      // [n_seq + 1]
  const int32_t* model_id;     // [n_seq]
  const int32_t* groups;       // [n_groups][LG_SB] sequence ids (one model per group), -1 empty
  int32_t n_groups;
  int32_t group_fill;          // most sequences in one group (1: the single-sequence cluster kernel)
  ModelView mv;
  float* fv;                   // [total_T][NP] forward vectors
  float* bv;                   // [total_T][NP] backward vectors (before the emission)
  double* oa;                  // [total_T] log2 offsets of fv rows
  double* ob;                  // [total_T] log2 offsets of bv rows
  // Viterbi
  uint16_t* psi;               // [total_T][NP] backpointers (cluster kernels)
  float* drow;                 // [total_T][NP] normalised delta rows (grouped kernel)
  float* logAT;                // [M][NP][NP] ln a transposed (grouped kernel's traceback)
  int32_t* path;               // [total_T]
  double* score;               // [n_seq]
  int* status;                 // device status word (bounded waits)
};

__device__ __forceinline__ float warp_max_f(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Group metadata in shared memory.
struct LgMeta {
  int64_t base[LG_SB];
  int len[LG_SB];
  int seq[LG_SB];
  int m, tmax;
};

__device__ inline void lg_load_meta(const LargeArgs& a, int g, LgMeta& md) {
  if (threadIdx.x == 0) {
    int tmax = 0, m = 0;
    for (int b = 0; b < LG_SB; ++b) {
      const int s = a.groups[(size_t)g * LG_SB + b];
      md.seq[b] = s;
      if (s >= 0) {
        md.base[b] = a.offsets[s];
        md.len[b] = (int)(a.offsets[s + 1] - a.offsets[s]);
        m = a.model_id[s];
      } else {
        md.base[b] = 0;
        md.len[b] = 0;
      }
      tmax = max(tmax, md.len[b]);
    }
    md.m = m;
    md.tmax = tmax;
  }
  __syncthreads();
}

// Forward (blockIdx.y == 0) and backward (1) recursions of one group.
template <int NP>
__global__ void __launch_bounds__(LG_NT) large_fb_kernel(LargeArgs a) {
  using S = LgShape<NP>;
  extern __shared__ __align__(16) float lsm[];
  __shared__ LgMeta md;
  float* vbuf = lsm;                                   // [2][LG_SB][NP]
  float* red = vbuf + 2 * LG_SB * NP;                  // [warps][LG_SB]
  float* As = red + (LG_NT / 32) * LG_SB;              // [NP][NP] (A_SMEM)
  const int dir = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cg = tid % S::CG, ts = tid / S::CG;
  const int N = a.mv.N;
  lg_load_meta(a, blockIdx.x, md);
  const int m = md.m;
  const float* Mg = (dir == 0 ? a.mv.A32 : a.mv.AT32) + (size_t)m * NP * NP;
  const float* Mp = Mg;
  if constexpr (S::A_SMEM) {
    for (int z = tid * 4; z < NP * NP; z += LG_NT * 4)
      *reinterpret_cast<float4*>(As + z) = __ldg(reinterpret_cast<const float4*>(Mg + z));
    Mp = As;
  }
  float* v0 = vbuf;
  float* v1 = vbuf + LG_SB * NP;
  double O[S::SBT];
#pragma unroll
  for (int r = 0; r < S::SBT; ++r) O[r] = 0.0;
  __syncthreads();

  for (int k = 0; k < md.tmax; ++k) {
    // emissions of this step (issued before the mat-vec to overlap latency)
    float lb[S::SBT][S::JC];
    int64_t row[S::SBT];
    bool act[S::SBT];
#pragma unroll
    for (int r = 0; r < S::SBT; ++r) {
      const int b = ts * S::SBT + r;
      act[r] = k < md.len[b];
      const int t = dir == 0 ? k : md.len[b] - 1 - k;
      row[r] = md.base[b] + t;
#pragma unroll
      for (int c = 0; c < S::JC; ++c) {
        const int j = cg + c * S::CG;
        lb[r][c] = (act[r] && j < N) ? __ldg(a.logb + row[r] * N + j) * kLog2ef : -INFINITY;
      }
    }
    float u[S::SBT][S::JC];
    if (k == 0) {
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) {
          const int j = cg + c * S::CG;
          if (dir == 0) {
            u[r][c] = lb[r][c] + a.mv.logpi2[(size_t)m * NP + j];
          } else {
            u[r][c] = lb[r][c];
            if (act[r]) a.bv[row[r] * NP + j] = j < N ? 1.f : 0.f;
          }
        }
      if (dir == 1 && cg == 0) {
#pragma unroll
        for (int r = 0; r < S::SBT; ++r)
          if (act[r]) a.ob[row[r]] = 0.0;
      }
    } else {
      float acc[S::SBT][S::JC];
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) acc[r][c] = 0.f;
      const float* vp = v0 + ts * S::SBT * NP;
#pragma unroll 2
      for (int i = 0; i < NP; i += 4) {
        float am[4][S::JC];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int c = 0; c < S::JC; ++c) {
            const float* p = Mp + (size_t)(i + q) * NP + cg + c * S::CG;
            am[q][c] = S::A_SMEM ? *p : __ldg(p);
          }
#pragma unroll
        for (int r = 0; r < S::SBT; ++r) {
          const float4 x = *reinterpret_cast<const float4*>(vp + r * NP + i);
#pragma unroll
          for (int c = 0; c < S::JC; ++c) {
            acc[r][c] = fmaf(x.x, am[0][c], acc[r][c]);
            acc[r][c] = fmaf(x.y, am[1][c], acc[r][c]);
            acc[r][c] = fmaf(x.z, am[2][c], acc[r][c]);
            acc[r][c] = fmaf(x.w, am[3][c], acc[r][c]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) {
          const int j = cg + c * S::CG;
          if (dir == 1 && act[r]) a.bv[row[r] * NP + j] = acc[r][c];
          u[r][c] = lb[r][c] + log2f(acc[r][c]);
        }
      if (dir == 1 && cg == 0) {
#pragma unroll
        for (int r = 0; r < S::SBT; ++r)
          if (act[r]) a.ob[row[r]] = O[r];
      }
    }
    // E = floor(max_j u_j) per sequence
#pragma unroll
    for (int r = 0; r < S::SBT; ++r) {
      float mx = -INFINITY;
#pragma unroll
      for (int c = 0; c < S::JC; ++c) mx = fmaxf(mx, u[r][c]);
      mx = warp_max_f(mx);
      if (lane == 0) red[warp * LG_SB + r] = mx;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < S::SBT; ++r) {
      float mx = -INFINITY;
#pragma unroll
      for (int w = 0; w < S::WPS; ++w) mx = fmaxf(mx, red[(ts * S::WPS + w) * LG_SB + r]);
      const float E = mx > -INFINITY ? floorf(mx) : 0.f;
      O[r] = (k == 0 ? 0.0 : O[r]) + (double)E;
      const int b = ts * S::SBT + r;
#pragma unroll
      for (int c = 0; c < S::JC; ++c) {
        const int j = cg + c * S::CG;
        const float v = exp2f(u[r][c] - E);
        v1[b * NP + j] = v;
        if (dir == 0 && act[r]) a.fv[row[r] * NP + j] = v;
      }
      if (dir == 0 && cg == 0 && act[r]) a.oa[row[r]] = O[r];
    }
    __syncthreads();
    float* tmp = v0;
    v0 = v1;
    v1 = tmp;
  }
}

// Max-plus recursion (Eq. 3-4) of one group with the operation order of the
// float32-mode reading: c = delta(i) + ln a_ij, delta_t(j) = max_i c + ln b_j(t),
// then the step maximum is subtracted and added to a float64 score offset.
// The recursion keeps values only (one add and one maximum per candidate)
// and stores every step's normalised row d_t [total_T][NP] (float32); the
// traceback recomputes the one backpointer it needs per step,
// psi_t(q_t) = the lowest i attaining max_i d_{t-1}(i) + ln a_{i q_t}, from
// the same float32 operands, which is what an upward strict-'>' scan gives.
// One warp per sequence of the group walks its path.
template <int NP>
struct LgVitShape {
  static constexpr size_t smem_bytes() {
    return (size_t)(3 * LG_SB * NP + (LG_NT / 32) * LG_SB) * 4 + (LgShape<NP>::A_SMEM ? (size_t)NP * NP * 4 : 0);
  }
};

template <int NP>
__global__ void __launch_bounds__(LG_NT) large_viterbi_kernel(LargeArgs a) {
  using S = LgShape<NP>;
  extern __shared__ __align__(16) float lsm[];
  __shared__ LgMeta md;
  __shared__ double soff[LG_SB];
  __shared__ int sidx[LG_NT / 32];
  float* vbuf = lsm;                                   // [2][LG_SB][NP]
  float* dfin = vbuf + 2 * LG_SB * NP;                 // [LG_SB][NP] last row of each sequence
  float* red = dfin + LG_SB * NP;                      // [warps][LG_SB]
  float* As = red + (LG_NT / 32) * LG_SB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cg = tid % S::CG, ts = tid / S::CG;
  const int N = a.mv.N;
  lg_load_meta(a, blockIdx.x, md);
  const int m = md.m;
  const float* Mg = a.mv.logAe + (size_t)m * NP * NP;
  const float* Mp = Mg;
  if constexpr (S::A_SMEM) {
    for (int z = tid * 4; z < NP * NP; z += LG_NT * 4)
      *reinterpret_cast<float4*>(As + z) = __ldg(reinterpret_cast<const float4*>(Mg + z));
    Mp = As;
  }
  float* d0 = vbuf;
  float* d1 = vbuf + LG_SB * NP;
  double off[S::SBT];
#pragma unroll
  for (int r = 0; r < S::SBT; ++r) off[r] = 0.0;
  __syncthreads();

  for (int k = 0; k < md.tmax; ++k) {
    float lb[S::SBT][S::JC], dn[S::SBT][S::JC];
    int64_t row[S::SBT];
    bool act[S::SBT];
#pragma unroll
    for (int r = 0; r < S::SBT; ++r) {
      const int b = ts * S::SBT + r;
      act[r] = k < md.len[b];
      row[r] = md.base[b] + k;
#pragma unroll
      for (int c = 0; c < S::JC; ++c) {
        const int j = cg + c * S::CG;
        lb[r][c] = (act[r] && j < N) ? __ldg(a.logb + row[r] * N + j) : -INFINITY;
      }
    }
    if (k == 0) {
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) dn[r][c] = a.mv.logpie[(size_t)m * NP + cg + c * S::CG] + lb[r][c];
    } else {
      // candidates in 8-row blocks of A, the next block's rows loaded while the
      // current one is used; adds two rows per instruction, two running maxima
      // per (sequence, column) (the maximum does not depend on the order)
      float b0[S::SBT][S::JC], b1[S::SBT][S::JC];
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) b0[r][c] = -INFINITY, b1[r][c] = -INFINITY;
      const float* dp = d0 + ts * S::SBT * NP;
      auto load8 = [&](float2 (&am)[4][S::JC], int i) {
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2)
#pragma unroll
          for (int c = 0; c < S::JC; ++c) {
            const float* p = Mp + (size_t)(i + 2 * q2) * NP + cg + c * S::CG;
            am[q2][c] = S::A_SMEM ? make_float2(p[0], p[NP]) : make_float2(__ldg(p), __ldg(p + NP));
          }
      };
      auto comp8 = [&](const float2 (&am)[4][S::JC], int i) {
#pragma unroll
        for (int r = 0; r < S::SBT; ++r) {
          const float4 x0 = *reinterpret_cast<const float4*>(dp + r * NP + i);
          const float4 x1 = *reinterpret_cast<const float4*>(dp + r * NP + i + 4);
          const float2 xv[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(x1.x, x1.y),
                                make_float2(x1.z, x1.w)};
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2)
#pragma unroll
            for (int c = 0; c < S::JC; ++c) {
              const float2 cc = __fadd2_rn(xv[q2], am[q2][c]);
              b0[r][c] = fmaxf(b0[r][c], cc.x);
              b1[r][c] = fmaxf(b1[r][c], cc.y);
            }
        }
      };
      float2 amA[4][S::JC], amB[4][S::JC];
      load8(amA, 0);
      for (int i = 0; i < NP; i += 16) {
        load8(amB, i + 8);
        comp8(amA, i);
        if (i + 16 < NP) load8(amA, i + 16);
        comp8(amB, i + 8);
      }
      float best[S::SBT][S::JC];
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) best[r][c] = fmaxf(b0[r][c], b1[r][c]);
#pragma unroll
      for (int r = 0; r < S::SBT; ++r)
#pragma unroll
        for (int c = 0; c < S::JC; ++c) dn[r][c] = best[r][c] + lb[r][c];
    }
#pragma unroll
    for (int r = 0; r < S::SBT; ++r) {
      float mx = -INFINITY;
#pragma unroll
      for (int c = 0; c < S::JC; ++c) mx = fmaxf(mx, dn[r][c]);
      mx = warp_max_f(mx);
      if (lane == 0) red[warp * LG_SB + r] = mx;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < S::SBT; ++r) {
      float mx = -INFINITY;
#pragma unroll
      for (int w = 0; w < S::WPS; ++w) mx = fmaxf(mx, red[(ts * S::WPS + w) * LG_SB + r]);
      const bool fin = mx > -INFINITY && mx < INFINITY;
      if (fin) off[r] += (double)mx;
      const int b = ts * S::SBT + r;
      const bool last = act[r] && k == md.len[b] - 1;
#pragma unroll
      for (int c = 0; c < S::JC; ++c) {
        const float d = fin ? dn[r][c] - mx : dn[r][c];
        d1[b * NP + cg + c * S::CG] = d;
        if (act[r]) a.drow[row[r] * NP + cg + c * S::CG] = d;
        if (last) dfin[b * NP + cg + c * S::CG] = d;
      }
      if (last && cg == 0) soff[b] = off[r];
    }
    __syncthreads();
    float* tmp = d0;
    d0 = d1;
    d1 = tmp;
  }

  // final states (the lowest index attaining the maximum of the last row)
  __shared__ int qfin[LG_SB];
  for (int b = 0; b < LG_SB; ++b) {
    const int s = md.seq[b], T = md.len[b];
    if (s < 0) continue;
    if (T == 0) {
      if (tid == 0) a.score[s] = 0.0;
      continue;
    }
    float mx = -INFINITY;
    for (int j = tid; j < NP; j += LG_NT) mx = fmaxf(mx, dfin[b * NP + j]);
    mx = warp_max_f(mx);
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = -INFINITY;
    for (int w = 0; w < LG_NT / 32; ++w) mx = fmaxf(mx, red[w]);
    int lo = NP;
    for (int j = tid; j < NP; j += LG_NT)
      if (dfin[b * NP + j] == mx && j < lo) lo = j;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    if (lane == 0) sidx[warp] = lo;
    __syncthreads();
    int q = NP;
    for (int w = 0; w < LG_NT / 32; ++w) q = min(q, sidx[w]);
    if (q >= NP) q = 0;   // every entry -inf: state 0, as the oracle's argmax
    if (tid == 0) {
      const float d = dfin[b * NP + q];
      a.score[s] = d > -INFINITY ? soff[b] + (double)d : -INFINITY;
      qfin[b] = q;
    }
    __syncthreads();
  }
  // tracebacks, warp b on sequence b: lane l scans rows i = l + 32 m upward
  // (strict '>'), the warp keeps the largest value and, among equal values,
  // the lowest index.  The next step's row d_{t-2} is loaded while step t is
  // reduced; ln a_{i q} is read as row q of the transposed table.
  static_assert(LG_NT / 32 == LG_SB, "one warp per sequence of the group");
  constexpr int PL = NP / 32;   // rows per lane
  {
    const int b = warp, s = md.seq[b], T = md.len[b];
    if (s >= 0 && T > 0) {
      const int64_t base = md.base[b];
      const float* AT = a.logAT + (size_t)m * NP * NP;
      int q = qfin[b];
      if (lane == 0) a.path[base + T - 1] = q;
      float dr[PL];
      if (T > 1) {
#pragma unroll
        for (int p = 0; p < PL; ++p) dr[p] = a.drow[(base + T - 2) * NP + lane + 32 * p];
      }
      for (int t = T - 1; t > 0; --t) {
        float cur[PL];
#pragma unroll
        for (int p = 0; p < PL; ++p) cur[p] = dr[p];
        if (t > 1) {
#pragma unroll
          for (int p = 0; p < PL; ++p) dr[p] = a.drow[(base + t - 2) * NP + lane + 32 * p];
        }
        const float* arow = AT + (size_t)q * NP;
        float bv = -INFINITY;
        int bi = 0;
#pragma unroll
        for (int p = 0; p < PL; ++p) {
          const float c = cur[p] + __ldg(arow + lane + 32 * p);
          if (c > bv) {
            bv = c;
            bi = lane + 32 * p;
          }
        }
        const float wv = warp_max_f(bv);
        int wi = bv == wv ? bi : NP;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wi = min(wi, __shfl_xor_sync(0xffffffffu, wi, o));
        q = wi >= NP ? 0 : wi;
        if (lane == 0) a.path[base + t - 1] = q;
      }
    }
  }
}

}  // namespace hmm
