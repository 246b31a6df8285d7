// Large-N recursions for few sequences at padded N = 256: a cluster of two
// CTAs per group (and direction) keeps the whole transition matrix resident
// in shared memory as float32 (each CTA its 128 columns, 128 KB), instead of
// one block re-reading 256 KB of A from L2 at every step.  This is the
// latency path of single long sequences (the request server, short batches):
// the steps of one sequence are sequential, so what counts is the time of
// one step, and the per-step mat-vec then runs from shared memory over 512
// threads.
//
// Per step of the forward (Eq. 1-2) / backward recursion in the shifted
// exp-space form of the large-N kernels (the same rows, offsets and
// semantics as large_fb_kernel, so the posterior / statistics / xi kernels
// are shared):
//   1. thread (c, h) of CTA r sums rows i in half h of column j = 128 r + c
//      of A^T v (backward: A z) for every sequence of the group, the two
//      halves are added in shared memory;
//   2. u = log2 b + log2 s for the CTA's 128 columns, the CTA's row maximum;
//   3. u and the row maximum go to both CTAs' shared memory (DSMEM stores),
//      then one cluster barrier (release / acquire);
//   4. every CTA forms E = floor(max) and the whole next vector
//      v = 2^(u - E) from both halves, and writes its own columns' rows.
// The Viterbi kernel runs the max-plus recursion (Eq. 3-4) the same way with
// the float32-mode operation order of large_viterbi_kernel: candidates
// delta(i) + ln a_ij scanned upward with a strict '>' (the two halves of i
// are joined keeping the lower half on ties, which is that scan), the step
// maximum subtracted and added to a float64 offset; CTA 0 traces back.
// Both kernels run the same number of cluster barriers in every CTA (the
// group's longest sequence), so the barriers always complete.
#include "launch.h"
#include "tc_common.cuh"

namespace hmm {
namespace {

using tc::cluster_rank;
using tc::cluster_sync;
using tc::mapa;
using tc::smem_u32;

constexpr int CL_NP = 256, CL_N = 2, CL_CW = CL_NP / CL_N, CL_NT = 256;

struct ClSmem {
  float As[CL_NP * CL_CW];          // A^T (forward) / A (backward) columns of this CTA: [i][c]
  float vfull[LG_SB * CL_NP];       // the whole previous vector of every sequence
  float ubuf[2][LG_SB * CL_NP];     // u (or delta) of both CTAs, double-buffered by step parity
  float mbuf[2][CL_N][LG_SB];       // the CTAs' row maxima
  float red[LG_SB * CL_CW];         // the upper half's partial sums
  int rarg[LG_SB * CL_CW];          // Viterbi: the upper half's arguments
  float wmax[CL_NT / 32][LG_SB];
  float dfin[LG_SB * CL_NP];        // Viterbi: last row of each sequence
  double soff[LG_SB];
};

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// u (or delta) value and row maximum of this CTA to both CTAs of the cluster
__device__ __forceinline__ void publish(ClSmem& sm, int par, int b, int j, float u, uint32_t rank) {
  const uint32_t a = smem_u32(&sm.ubuf[par][b * CL_NP + j]);
#pragma unroll
  for (uint32_t q = 0; q < CL_N; ++q) st_cluster_f32(mapa(a, q), u);
  (void)rank;
}

__device__ __forceinline__ void load_group(const LargeArgs& a, int g, LgMeta& md) {
  if (threadIdx.x == 0) {
    int tmax = 0, m = 0;
    for (int b = 0; b < LG_SB; ++b) {
      const int s = a.groups[(size_t)g * LG_SB + b];
      md.seq[b] = s;
      md.base[b] = s >= 0 ? a.offsets[s] : 0;
      md.len[b] = s >= 0 ? (int)(a.offsets[s + 1] - a.offsets[s]) : 0;
      if (s >= 0) m = a.model_id[s];
      tmax = max(tmax, md.len[b]);
    }
    md.m = m;
    md.tmax = tmax;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(CL_NT, 1) large_fb_cl_kernel(LargeArgs a) {
  extern __shared__ __align__(16) unsigned char cl_raw[];
  ClSmem& sm = *reinterpret_cast<ClSmem*>(cl_raw);
  __shared__ LgMeta md;
  const uint32_t rank = cluster_rank();
  const int g = blockIdx.y, dir = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = tid % CL_CW, h = tid / CL_CW;       // column of this CTA, half of the sum
  const int j = (int)rank * CL_CW + c;               // output state of this thread
  const int N = a.mv.N;
  load_group(a, g, md);
  const int m = md.m;
  const float* Mg = (dir == 0 ? a.mv.A32 : a.mv.AT32) + (size_t)m * CL_NP * CL_NP;
  for (int z = tid; z < CL_NP * CL_CW; z += CL_NT) {
    const int i = z / CL_CW, cc = z % CL_CW;
    sm.As[z] = __ldg(Mg + (size_t)i * CL_NP + rank * CL_CW + cc);
  }
  int nb = 0;
  for (int b = 0; b < LG_SB; ++b)
    if (md.seq[b] >= 0) nb = b + 1;
  double O[LG_SB];
#pragma unroll
  for (int b = 0; b < LG_SB; ++b) O[b] = 0.0;
  __syncthreads();
  cluster_sync();   // both CTAs resident before any DSMEM store

  for (int k = 0; k < md.tmax; ++k) {
    const int par = k & 1;
    // emissions of the owned column (lower-half threads), issued first
    float lb[LG_SB];
    int64_t row[LG_SB];
#pragma unroll
    for (int b = 0; b < LG_SB; ++b) {
      const bool act = b < nb && k < md.len[b];
      const int t = dir == 0 ? k : md.len[b] - 1 - k;
      row[b] = md.base[b] + t;
      lb[b] = (h == 0 && act && j < N) ? __ldg(a.logb + row[b] * N + j) * kLog2ef : -INFINITY;
    }
    float s[LG_SB];
    if (k > 0) {
      float acc[LG_SB][4];
#pragma unroll
      for (int b = 0; b < LG_SB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[b][q] = 0.f;
      const int i0 = h * (CL_NP / 2);
#pragma unroll 4
      for (int i = i0; i < i0 + CL_NP / 2; i += 4) {
        const float a0 = sm.As[(i + 0) * CL_CW + c], a1 = sm.As[(i + 1) * CL_CW + c];
        const float a2 = sm.As[(i + 2) * CL_CW + c], a3 = sm.As[(i + 3) * CL_CW + c];
#pragma unroll
        for (int b = 0; b < LG_SB; ++b) {
          if (b < nb) {
            const float4 x = *reinterpret_cast<const float4*>(&sm.vfull[b * CL_NP + i]);
            acc[b][0] = fmaf(x.x, a0, acc[b][0]);
            acc[b][1] = fmaf(x.y, a1, acc[b][1]);
            acc[b][2] = fmaf(x.z, a2, acc[b][2]);
            acc[b][3] = fmaf(x.w, a3, acc[b][3]);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < LG_SB; ++b) {
        s[b] = (acc[b][0] + acc[b][1]) + (acc[b][2] + acc[b][3]);
        if (h == 1) sm.red[b * CL_CW + c] = s[b];
      }
    }
    __syncthreads();
    float u[LG_SB];
#pragma unroll
    for (int b = 0; b < LG_SB; ++b) {
      const bool act = b < nb && k < md.len[b];
      if (k == 0) {
        u[b] = dir == 0 ? lb[b] + a.mv.logpi2[(size_t)m * CL_NP + j] : lb[b];
        if (h == 0 && dir == 1 && act) a.bv[row[b] * CL_NP + j] = j < N ? 1.f : 0.f;
      } else {
        const float sj = s[b] + sm.red[b * CL_CW + c];
        if (h == 0 && dir == 1 && act) a.bv[row[b] * CL_NP + j] = sj;
        u[b] = lb[b] + log2f(sj);
      }
      float mx = h == 0 ? u[b] : -INFINITY;
      mx = warp_max_f(mx);
      if (lane == 0) sm.wmax[warp][b] = mx;
    }
    if (dir == 1 && rank == 0 && tid == 0)
      for (int b = 0; b < nb; ++b)
        if (k < md.len[b]) a.ob[row[b]] = k == 0 ? 0.0 : O[b];
    __syncthreads();
    if (h == 0) {
      for (int b = 0; b < nb; ++b) publish(sm, par, b, j, u[b], rank);
    } else if (tid - CL_CW < LG_SB) {
      const int b = tid - CL_CW;
      float mx = -INFINITY;
      for (int w = 0; w < CL_CW / 32; ++w) mx = fmaxf(mx, sm.wmax[w][b]);
      const uint32_t ad = smem_u32(&sm.mbuf[par][rank][b]);
      for (uint32_t q = 0; q < CL_N; ++q) st_cluster_f32(mapa(ad, q), mx);
    }
    cluster_sync();
    // E, offsets and the whole next vector
#pragma unroll
    for (int b = 0; b < LG_SB; ++b) {
      if (b >= nb) continue;
      float mx = -INFINITY;
#pragma unroll
      for (int q = 0; q < CL_N; ++q) mx = fmaxf(mx, sm.mbuf[par][q][b]);
      const float E = mx > -INFINITY ? floorf(mx) : 0.f;
      O[b] = (k == 0 ? 0.0 : O[b]) + (double)E;
      const bool act = k < md.len[b];
      for (int z = tid; z < CL_NP; z += CL_NT) {
        const float v = exp2f(sm.ubuf[par][b * CL_NP + z] - E);
        sm.vfull[b * CL_NP + z] = v;
        if (dir == 0 && act && (z / CL_CW) == (int)rank) a.fv[row[b] * CL_NP + z] = v;
      }
      if (dir == 0 && act && rank == 0 && tid == 0) a.oa[row[b]] = O[b];
    }
    __syncthreads();
  }
  cluster_sync();   // no CTA leaves while its peer may still store into it
}

__global__ void __launch_bounds__(CL_NT, 1) large_vit_cl_kernel(LargeArgs a) {
  extern __shared__ __align__(16) unsigned char cl_raw[];
  ClSmem& sm = *reinterpret_cast<ClSmem*>(cl_raw);
  __shared__ LgMeta md;
  __shared__ int sidx[CL_NT / 32];
  const uint32_t rank = cluster_rank();
  const int g = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = tid % CL_CW, h = tid / CL_CW;
  const int j = (int)rank * CL_CW + c;
  const int N = a.mv.N;
  load_group(a, g, md);
  const int m = md.m;
  const float* Mg = a.mv.logAe + (size_t)m * CL_NP * CL_NP;
  for (int z = tid; z < CL_NP * CL_CW; z += CL_NT) {
    const int i = z / CL_CW, cc = z % CL_CW;
    sm.As[z] = __ldg(Mg + (size_t)i * CL_NP + rank * CL_CW + cc);
  }
  int nb = 0;
  for (int b = 0; b < LG_SB; ++b)
    if (md.seq[b] >= 0) nb = b + 1;
  double off[LG_SB];
#pragma unroll
  for (int b = 0; b < LG_SB; ++b) off[b] = 0.0;
  __syncthreads();
  cluster_sync();

  for (int k = 0; k < md.tmax; ++k) {
    const int par = k & 1;
    float lb[LG_SB];
    int64_t row[LG_SB];
#pragma unroll
    for (int b = 0; b < LG_SB; ++b) {
      const bool act = b < nb && k < md.len[b];
      row[b] = md.base[b] + k;
      lb[b] = (h == 0 && act && j < N) ? __ldg(a.logb + row[b] * N + j) : -INFINITY;
    }
    float best[LG_SB];
    int arg[LG_SB];
    if (k > 0) {
#pragma unroll
      for (int b = 0; b < LG_SB; ++b) best[b] = -INFINITY, arg[b] = 0;
      const int i0 = h * (CL_NP / 2);
      for (int i = i0; i < i0 + CL_NP / 2; i += 4) {
        const float a0 = sm.As[(i + 0) * CL_CW + c], a1 = sm.As[(i + 1) * CL_CW + c];
        const float a2 = sm.As[(i + 2) * CL_CW + c], a3 = sm.As[(i + 3) * CL_CW + c];
#pragma unroll
        for (int b = 0; b < LG_SB; ++b) {
          if (b < nb) {
            const float4 x = *reinterpret_cast<const float4*>(&sm.vfull[b * CL_NP + i]);
            const float cv[4] = {x.x + a0, x.y + a1, x.z + a2, x.w + a3};
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (cv[q] > best[b]) {
                best[b] = cv[q];
                arg[b] = i + q;
              }
          }
        }
      }
#pragma unroll
      for (int b = 0; b < LG_SB; ++b)
        if (h == 1) {
          sm.red[b * CL_CW + c] = best[b];
          sm.rarg[b * CL_CW + c] = arg[b];
        }
    }
    __syncthreads();
    float dn[LG_SB];
#pragma unroll
    for (int b = 0; b < LG_SB; ++b) {
      const bool act = b < nb && k < md.len[b];
      if (k == 0) {
        dn[b] = a.mv.logpie[(size_t)m * CL_NP + j] + lb[b];
      } else {
        // the upper half of i wins only when strictly larger: the upward scan
        float bv = best[b];
        int ba = arg[b];
        const float bu = sm.red[b * CL_CW + c];
        if (bu > bv) {
          bv = bu;
          ba = sm.rarg[b * CL_CW + c];
        }
        dn[b] = bv + lb[b];
        if (h == 0 && act) a.psi[row[b] * CL_NP + j] = (uint16_t)ba;
      }
      float mx = h == 0 ? dn[b] : -INFINITY;
      mx = warp_max_f(mx);
      if (lane == 0) sm.wmax[warp][b] = mx;
    }
    __syncthreads();
    if (h == 0) {
      for (int b = 0; b < nb; ++b) publish(sm, par, b, j, dn[b], rank);
    } else if (tid - CL_CW < LG_SB) {
      const int b = tid - CL_CW;
      float mx = -INFINITY;
      for (int w = 0; w < CL_CW / 32; ++w) mx = fmaxf(mx, sm.wmax[w][b]);
      const uint32_t ad = smem_u32(&sm.mbuf[par][rank][b]);
      for (uint32_t q = 0; q < CL_N; ++q) st_cluster_f32(mapa(ad, q), mx);
    }
    cluster_sync();
#pragma unroll
    for (int b = 0; b < LG_SB; ++b) {
      if (b >= nb) continue;
      float mx = -INFINITY;
#pragma unroll
      for (int q = 0; q < CL_N; ++q) mx = fmaxf(mx, sm.mbuf[par][q][b]);
      const bool fin = mx > -INFINITY && mx < INFINITY;
      if (fin) off[b] += (double)mx;
      const bool last = k == md.len[b] - 1;
      for (int z = tid; z < CL_NP; z += CL_NT) {
        const float dv = sm.ubuf[par][b * CL_NP + z];
        const float d = fin ? dv - mx : dv;
        sm.vfull[b * CL_NP + z] = d;
        if (last) sm.dfin[b * CL_NP + z] = d;
      }
      if (last && tid == 0) sm.soff[b] = off[b];
    }
    __syncthreads();
  }
  __threadfence();   // every CTA's pointer rows are visible before the traceback
  cluster_sync();
  if (rank != 0) return;

  // final states and tracebacks (CTA 0), as large_viterbi_kernel
  uint16_t* stage = reinterpret_cast<uint16_t*>(sm.ubuf);
  constexpr int TB = LG_TB;
  for (int b = 0; b < LG_SB; ++b) {
    const int s = md.seq[b], T = md.len[b];
    if (s < 0) continue;
    if (T == 0) {
      if (tid == 0) a.score[s] = 0.0;
      continue;
    }
    float mx = -INFINITY;
    for (int z = tid; z < CL_NP; z += CL_NT) mx = fmaxf(mx, sm.dfin[b * CL_NP + z]);
    mx = warp_max_f(mx);
    if (lane == 0) sm.wmax[warp][0] = mx;
    __syncthreads();
    mx = -INFINITY;
    for (int w = 0; w < CL_NT / 32; ++w) mx = fmaxf(mx, sm.wmax[w][0]);
    int lo = CL_NP;
    for (int z = tid; z < CL_NP; z += CL_NT)
      if (sm.dfin[b * CL_NP + z] == mx && z < lo) lo = z;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    if (lane == 0) sidx[warp] = lo;
    __syncthreads();
    int q = CL_NP;
    for (int w = 0; w < CL_NT / 32; ++w) q = min(q, sidx[w]);
    if (q >= CL_NP) q = 0;
    if (tid == 0) {
      const float d = sm.dfin[b * CL_NP + q];
      a.score[s] = d > -INFINITY ? sm.soff[b] + (double)d : -INFINITY;
    }
    const int64_t base = md.base[b];
    int thi = T - 1;
    while (thi > 0) {
      const int tlo = max(0, thi - TB);
      const int rows = thi - tlo;
      __syncthreads();
      for (int z = tid; z < rows * CL_NP; z += CL_NT) stage[z] = a.psi[(base + tlo + 1) * CL_NP + z];
      __syncthreads();
      if (tid == 0) {
        for (int t = thi; t > tlo; --t) {
          a.path[base + t] = q;
          q = stage[(t - tlo - 1) * CL_NP + q];
        }
      }
      thi = tlo;
    }
    if (tid == 0) a.path[base] = q;
    __syncthreads();
  }
}

template <class K>
cudaError_t launch_cl(K kern, const LargeArgs& a, unsigned dirs, cudaStream_t st) {
  const size_t smem = sizeof(ClSmem);
  cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL_N, (unsigned)a.n_groups, dirs);
  cfg.blockDim = dim3(CL_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL_N;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

bool large_cl_supported(int NP, int n_groups) { return NP == CL_NP && n_groups > 0 && n_groups <= LG_CL_MAX_GROUPS; }

cudaError_t launch_large_fb_cl(const LargeArgs& a, cudaStream_t st) { return launch_cl(large_fb_cl_kernel, a, 2, st); }

cudaError_t launch_large_viterbi_cl(const LargeArgs& a, cudaStream_t st) {
  return launch_cl(large_vit_cl_kernel, a, 1, st);
}

}  // namespace hmm
