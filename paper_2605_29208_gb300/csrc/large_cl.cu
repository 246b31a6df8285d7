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

// ---------------------------------------------------------------------------
// One sequence per group (the request server's case: every request its own
// model).  Per step the mat-vec is 65,536 FMAs, so the step time is the
// latency of its dependency chain; this variant takes the cluster-wide
// barrier out of that chain.  Each CTA scales its columns by its own power of
// two E_r = floor(max of its u) and sends the scaled values v' and E_r to
// every CTA of the cluster with st.async stores that complete a transaction
// count on the receiver's mbarrier (two, by step parity); a receiver waits on
// its own mbarrier only.  The step's shift is E = max_r E_r = floor(max u)
// (floor is monotone), the shift of large_fb_kernel, and v = v' 2^(E_r - E)
// is applied as an exact power-of-two scaling of each CTA's part of the
// mat-vec and of the stored row.  The transition column block of a thread
// lives in registers (64 rows), the vector in shared memory; lanes 8q + c of
// a warp hold quarter q of the rows of column c, combined by shuffles.  One
// __syncthreads per step (the CTA's row maximum).
template <int NP_, int CLN>
struct Cl1 {
  static constexpr int NP = NP_;
  static constexpr int CW = NP / CLN;    // columns per CTA
  static constexpr int Q = 4;            // lanes per column (row quarters)
  static constexpr int RPT = NP / Q;     // rows per thread
  static constexpr int NW = CW / 8;      // warps per CTA (8 columns each)
  static constexpr int NT = NW * 32;
  static constexpr int VP = RPT + 4;     // padded quarter stride (bank offset)
  static constexpr uint32_t RX = (uint32_t)(CLN - 1) * (CW + 1) * 4;   // bytes received per step
  static_assert(CW % RPT == 0 || RPT % CW == 0, "a quarter must lie in one CTA's columns");
  static_assert(RPT % 4 == 0, "rows per thread in float4 blocks");
};

template <class S, int CLN>
struct Cl1Smem {
  float v[2][S::Q * S::VP];   // v' of every state (padded by quarter), by step parity
  float E[2][CLN];            // E_r of every CTA, by step parity
  float wmax[2][S::NW];       // warp maxima, by step parity
  uint64_t bar[2];            // completion of a step's vector, by parity
};

__device__ __forceinline__ void st_async_v4(uint32_t addr, float4 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(v), "r"(bar)
               : "memory");
}
// bounded wait with cluster-scope acquire (the data of st.async stores)
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* b, uint32_t parity) {
  const uint32_t addr = smem_u32(b);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, "
        "p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > tc::TC_WAIT_CYCLES) return false;
  }
}
// x 2^(Er - E) (0 for a CTA whose values are all zero)
__device__ __forceinline__ float cl1_scale(float x, float Er, float E) {
  return Er > -INFINITY ? ldexpf(x, (int)(Er - E)) : 0.f;
}
template <int RPT>
__device__ __forceinline__ int cl1_vidx(int j) { return j + 4 * (j / RPT); }

template <int NP_, int CLN>
__global__ void __launch_bounds__(Cl1<NP_, CLN>::NT, 1) large_fb_cl1_kernel(LargeArgs a) {
  using S = Cl1<NP_, CLN>;
  constexpr int NP = S::NP, CW = S::CW, RPT = S::RPT, NW = S::NW;
  __shared__ __align__(16) Cl1Smem<S, CLN> sm;
  const uint32_t rank = cluster_rank();
  const int g = blockIdx.y, dir = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c8 = lane & 7, q = lane >> 3;
  const int j = (int)rank * CW + warp * 8 + c8;     // state of this thread's column
  const int N = a.mv.N;
  const int s = a.groups[(size_t)g * LG_SB];
  const int64_t base = a.offsets[s];
  const int T = (int)(a.offsets[s + 1] - base);
  const int m = a.model_id[s];
  const int rq = (q * RPT) / CW;                    // CTA whose columns are this thread's rows
  const float* Mg = (dir == 0 ? a.mv.A32 : a.mv.AT32) + (size_t)m * NP * NP;
  float2 Ar[RPT / 2];
#pragma unroll
  for (int p = 0; p < RPT / 2; ++p)
    Ar[p] = make_float2(__ldg(Mg + (size_t)(q * RPT + 2 * p) * NP + j), __ldg(Mg + (size_t)(q * RPT + 2 * p + 1) * NP + j));
  if (tid == 0) {
    tc::mbar_init(&sm.bar[0], 2 * NW + 2);
    tc::mbar_init(&sm.bar[1], 2 * NW + 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    tc::mbar_expect_tx(&sm.bar[0], S::RX);
    if (T > 1) tc::mbar_expect_tx(&sm.bar[1], S::RX);
  }
  cluster_sync();   // every CTA's barriers initialised before any remote store

  auto tof = [&](int k) { return dir == 0 ? k : T - 1 - k; };
  // emissions two steps ahead in a register pair (the loop runs two steps per
  // pass), raw loads from a clamped row so that nothing waits on them early
  const int jc = min(j, N - 1);
  auto lbraw = [&](int k) { return __ldg(a.logb + (base + tof(min(k, T - 1))) * N + jc); };
  float lbA = 0.f, lbB = 0.f;
  if (T > 0) {
    lbA = lbraw(0);
    lbB = lbraw(1);
  }
  double O = 0.0;            // log2 offset after the previous step (thread 0)
  bool dead = false;
  float vprev = 0.f, Eprev = 0.f;
  int64_t rowprev = 0;
  auto step = [&](const int k, float& lbr) {
    const int par = k & 1;
    const int64_t row = base + tof(k);
    const float lb_cur = j < N ? lbr * kLog2ef : -INFINITY;
    if (k + 2 < T) lbr = lbraw(k + 2);
    float u;
    if (k == 0) {
      u = dir == 0 ? lb_cur + a.mv.logpi2[(size_t)m * NP + j] : lb_cur;
      if (dir == 1 && q == 0) a.bv[row * NP + j] = j < N ? 1.f : 0.f;
      if (dir == 1 && rank == 0 && tid == 0) a.ob[row] = 0.0;
    } else {
      const int pp = par ^ 1;
      if (!dead && !mbar_wait_cl(&sm.bar[pp], (uint32_t)((k - 1) >> 1) & 1u)) {
        set_status(a.status, ST_TIMEOUT);
        dead = true;   // the protocol is broken: finish without waiting (results invalid, status set)
      }
      if (tid == 0 && k + 1 < T) tc::mbar_expect_tx(&sm.bar[pp], S::RX);   // its phase of step k + 1
      float Er[CLN], E = -INFINITY;
#pragma unroll
      for (int r = 0; r < CLN; ++r) {
        Er[r] = sm.E[pp][r];
        E = fmaxf(E, Er[r]);
      }
      if (!(E > -INFINITY)) E = 0.f;
      if (tid == 0) O += (double)E;
      if (dir == 0) {   // the previous step's row, now that its shift is known
        if (q == 0) a.fv[rowprev * NP + j] = cl1_scale(vprev, Eprev, E);
        if (rank == 0 && tid == 0) a.oa[rowprev] = O;
      }
      const float* vb = &sm.v[pp][q * S::VP];
      float2 acc[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < RPT / 4; ++p) {
        const float4 x = *reinterpret_cast<const float4*>(vb + 4 * p);
        acc[2 * (p & 1)] = __ffma2_rn(make_float2(x.x, x.y), Ar[2 * p], acc[2 * (p & 1)]);
        acc[2 * (p & 1) + 1] = __ffma2_rn(make_float2(x.z, x.w), Ar[2 * p + 1], acc[2 * (p & 1) + 1]);
      }
      const float2 acc0 = make_float2(acc[0].x + acc[2].x, acc[0].y + acc[2].y);
      const float2 acc1 = make_float2(acc[1].x + acc[3].x, acc[1].y + acc[3].y);
      float Erq = Er[0];
#pragma unroll
      for (int r = 1; r < CLN; ++r)
        if (r == rq) Erq = Er[r];
      float part = cl1_scale((acc0.x + acc0.y) + (acc1.x + acc1.y), Erq, E);
      part += __shfl_xor_sync(0xffffffffu, part, 8);
      part += __shfl_xor_sync(0xffffffffu, part, 16);
      if (dir == 1) {
        if (q == 0) a.bv[row * NP + j] = part;
        if (rank == 0 && tid == 0) a.ob[row] = O;
      }
      u = lb_cur + log2f(part);
    }
    float mx = u;
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
    if (lane == 0) sm.wmax[par][warp] = mx;
    __syncthreads();
    float cm = -INFINITY;
#pragma unroll
    for (int w = 0; w < NW; ++w) cm = fmaxf(cm, sm.wmax[par][w]);
    const float Eown = cm > -INFINITY ? floorf(cm) : -INFINITY;
    const float vj = Eown > -INFINITY ? exp2f(u - Eown) : 0.f;
    __syncwarp();
    // lanes c8 = 0 and 4 of quarter q send four consecutive columns to CTA q
    const float v1 = __shfl_down_sync(0xffffffffu, vj, 1);
    const float v2 = __shfl_down_sync(0xffffffffu, vj, 2);
    const float v3 = __shfl_down_sync(0xffffffffu, vj, 3);
    if ((c8 & 3) == 0 && q < CLN) {
      const float4 pk = make_float4(vj, v1, v2, v3);
      float* dst = &sm.v[par][cl1_vidx<RPT>(j)];
      if (q == (int)rank) {
        *reinterpret_cast<float4*>(dst) = pk;
        tc::mbar_arrive(&sm.bar[par]);
      } else {
        st_async_v4(mapa(smem_u32(dst), (uint32_t)q), pk, mapa(smem_u32(&sm.bar[par]), (uint32_t)q));
      }
    }
    if (warp == 0 && lane < CLN) {
      if (lane == (int)rank) {
        sm.E[par][rank] = Eown;
        tc::mbar_arrive(&sm.bar[par]);
      } else {
        st_async_f32(mapa(smem_u32(&sm.E[par][rank]), (uint32_t)lane), Eown,
                     mapa(smem_u32(&sm.bar[par]), (uint32_t)lane));
      }
    }
    vprev = vj;
    Eprev = Eown;
    rowprev = row;
  };
  for (int k = 0; k < T; k += 2) {
    step(k, lbA);
    if (k + 1 < T) step(k + 1, lbB);
  }
  if (T > 0) {   // the last step's vector: every incoming store has landed; forward: the last row
    const int pp = (T - 1) & 1;
    if (!dead && !mbar_wait_cl(&sm.bar[pp], (uint32_t)((T - 1) >> 1) & 1u)) set_status(a.status, ST_TIMEOUT);
    if (dir == 0) {
      float E = -INFINITY;
#pragma unroll
      for (int r = 0; r < CLN; ++r) E = fmaxf(E, sm.E[pp][r]);
      if (!(E > -INFINITY)) E = 0.f;
      if (q == 0) a.fv[rowprev * NP + j] = cl1_scale(vprev, Eprev, E);
      if (rank == 0 && tid == 0) a.oa[rowprev] = O + (double)E;
    }
  }
  cluster_sync();
}

// Viterbi for one sequence per group, the same exchange: each CTA sends its
// columns' raw delta_k (the candidates' maximum plus ln b, before the step's
// normalisation) and its maximum; a receiver takes the step maximum mx over
// the CTAs, subtracts it from the rows it scans (the float32-mode order of
// large_viterbi_kernel: (delta - mx) + ln a_ij, upward, strict '>'; the row
// quarters of a column are joined in order, the lower keeping ties) and adds
// mx to the float64 offset.  CTA 0 picks the final state and traces back.
template <int NP_, int CLN>
__global__ void __launch_bounds__(Cl1<NP_, CLN>::NT, 1) large_vit_cl1_kernel(LargeArgs a) {
  using S = Cl1<NP_, CLN>;
  constexpr int NP = S::NP, CW = S::CW, RPT = S::RPT, NW = S::NW, NT = S::NT;
  constexpr int TB = 32768 / (2 * NP);   // traceback rows staged per chunk (32 KB)
  __shared__ __align__(16) Cl1Smem<S, CLN> sm;
  __shared__ __align__(16) uint16_t stage[TB * NP];
  __shared__ int sidx[NW];
  const uint32_t rank = cluster_rank();
  const int g = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c8 = lane & 7, q = lane >> 3;
  const int j = (int)rank * CW + warp * 8 + c8;
  const int N = a.mv.N;
  const int s = a.groups[(size_t)g * LG_SB];
  const int64_t base = a.offsets[s];
  const int T = (int)(a.offsets[s + 1] - base);
  const int m = a.model_id[s];
  const float* Mg = a.mv.logAe + (size_t)m * NP * NP;
  float2 Ar[RPT / 2];
#pragma unroll
  for (int p = 0; p < RPT / 2; ++p)
    Ar[p] = make_float2(__ldg(Mg + (size_t)(q * RPT + 2 * p) * NP + j), __ldg(Mg + (size_t)(q * RPT + 2 * p + 1) * NP + j));
  if (tid == 0) {
    tc::mbar_init(&sm.bar[0], 2 * NW + 2);
    tc::mbar_init(&sm.bar[1], 2 * NW + 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    tc::mbar_expect_tx(&sm.bar[0], S::RX);
    if (T > 1) tc::mbar_expect_tx(&sm.bar[1], S::RX);
  }
  cluster_sync();

  const int jc = min(j, N - 1);
  auto lbraw = [&](int k) { return __ldg(a.logb + (base + min(k, T - 1)) * N + jc); };
  float lbA = 0.f, lbB = 0.f;
  if (T > 0) {
    lbA = lbraw(0);
    lbB = lbraw(1);
  }
  double off = 0.0;   // thread 0
  bool dead = false;
  auto step = [&](const int k, float& lbr) {
    const int par = k & 1;
    const int64_t row = base + k;
    const float lb_cur = j < N ? lbr : -INFINITY;
    if (k + 2 < T) lbr = lbraw(k + 2);
    float dn;
    if (k == 0) {
      dn = a.mv.logpie[(size_t)m * NP + j] + lb_cur;
    } else {
      const int pp = par ^ 1;
      if (!dead && !mbar_wait_cl(&sm.bar[pp], (uint32_t)((k - 1) >> 1) & 1u)) {
        set_status(a.status, ST_TIMEOUT);
        dead = true;
      }
      if (tid == 0 && k + 1 < T) tc::mbar_expect_tx(&sm.bar[pp], S::RX);
      float mx = -INFINITY;
#pragma unroll
      for (int r = 0; r < CLN; ++r) mx = fmaxf(mx, sm.E[pp][r]);
      const bool fin = mx > -INFINITY && mx < INFINITY;
      if (tid == 0 && fin) off += (double)mx;
      const float* vb = &sm.v[pp][q * S::VP];
      // four sub-ranges of the quarter scanned side by side (shorter chains),
      // then joined in order: a later sub-range only when strictly larger
      constexpr int PS = RPT / 16;   // float4 blocks per sub-range
      float bs[4];
      int as[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) bs[r] = -INFINITY, as[r] = 0;
      // x - mx as x + (-mx), and x + (-0) = x exactly when the step is not normalised
      const float2 neg = fin ? make_float2(-mx, -mx) : make_float2(-0.f, -0.f);
#pragma unroll
      for (int p = 0; p < RPT / 4; ++p) {
        const int r = p / PS;
        const float4 x = *reinterpret_cast<const float4*>(vb + 4 * p);
        const float2 c01 = __fadd2_rn(__fadd2_rn(make_float2(x.x, x.y), neg), Ar[2 * p]);
        const float2 c23 = __fadd2_rn(__fadd2_rn(make_float2(x.z, x.w), neg), Ar[2 * p + 1]);
        const float cv[4] = {c01.x, c01.y, c23.x, c23.y};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (cv[e] > bs[r]) {
            bs[r] = cv[e];
            as[r] = q * RPT + 4 * p + e;
          }
      }
      float best = bs[0];
      int arg = as[0];
#pragma unroll
      for (int r = 1; r < 4; ++r)
        if (bs[r] > best) best = bs[r], arg = as[r];
      // quarters in order: a later quarter wins only when strictly larger
      float bo = __shfl_down_sync(0xffffffffu, best, 8);
      int ao = __shfl_down_sync(0xffffffffu, arg, 8);
      if (bo > best) best = bo, arg = ao;
      bo = __shfl_down_sync(0xffffffffu, best, 16);
      ao = __shfl_down_sync(0xffffffffu, arg, 16);
      if (bo > best) best = bo, arg = ao;
      // lanes of quarter 0 hold the joined result; every lane takes its column's
      if (q == 0) a.psi[row * NP + j] = (uint16_t)arg;
      best = __shfl_sync(0xffffffffu, best, c8);
      dn = best + lb_cur;
    }
    float wm = dn;
    wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, 1));
    wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, 2));
    wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, 4));
    if (lane == 0) sm.wmax[par][warp] = wm;
    __syncthreads();
    float cm = -INFINITY;
#pragma unroll
    for (int w = 0; w < NW; ++w) cm = fmaxf(cm, sm.wmax[par][w]);
    __syncwarp();
    const float v1 = __shfl_down_sync(0xffffffffu, dn, 1);
    const float v2 = __shfl_down_sync(0xffffffffu, dn, 2);
    const float v3 = __shfl_down_sync(0xffffffffu, dn, 3);
    if ((c8 & 3) == 0 && q < CLN) {
      const float4 pk = make_float4(dn, v1, v2, v3);
      float* dst = &sm.v[par][cl1_vidx<RPT>(j)];
      if (q == (int)rank) {
        *reinterpret_cast<float4*>(dst) = pk;
        tc::mbar_arrive(&sm.bar[par]);
      } else {
        st_async_v4(mapa(smem_u32(dst), (uint32_t)q), pk, mapa(smem_u32(&sm.bar[par]), (uint32_t)q));
      }
    }
    if (warp == 0 && lane < CLN) {
      if (lane == (int)rank) {
        sm.E[par][rank] = cm;
        tc::mbar_arrive(&sm.bar[par]);
      } else {
        st_async_f32(mapa(smem_u32(&sm.E[par][rank]), (uint32_t)lane), cm, mapa(smem_u32(&sm.bar[par]), (uint32_t)lane));
      }
    }
  };
  for (int k = 0; k < T; k += 2) {
    step(k, lbA);
    if (k + 1 < T) step(k + 1, lbB);
  }
  if (T > 0) {
    const int pp = (T - 1) & 1;
    if (!dead && !mbar_wait_cl(&sm.bar[pp], (uint32_t)((T - 1) >> 1) & 1u)) set_status(a.status, ST_TIMEOUT);
  }
  __threadfence();   // every CTA's pointer rows are visible before the traceback
  cluster_sync();
  if (rank != 0) return;
  if (T == 0) {
    if (tid == 0) a.score[s] = 0.0;
    return;
  }
  // final state: the lowest index of the normalised last row's maximum
  const int pp = (T - 1) & 1;
  float mx = -INFINITY;
#pragma unroll
  for (int r = 0; r < CLN; ++r) mx = fmaxf(mx, sm.E[pp][r]);
  const bool fin = mx > -INFINITY && mx < INFINITY;
  if (tid == 0 && fin) off += (double)mx;
  float dz = -INFINITY;
  if (tid < NP) {
    const float x = sm.v[pp][cl1_vidx<RPT>(tid)];
    dz = fin ? x - mx : x;
  }
  float dmax = dz;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) sm.wmax[0][warp] = dmax;
  __syncthreads();
  dmax = -INFINITY;
  for (int w = 0; w < NW; ++w) dmax = fmaxf(dmax, sm.wmax[0][w]);
  int lo = (tid < NP && dz == dmax) ? tid : NP;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  if (lane == 0) sidx[warp] = lo;
  __syncthreads();
  int st = NP;
  for (int w = 0; w < NW; ++w) st = min(st, sidx[w]);
  if (st >= NP) st = 0;
  if (tid == 0) {
    const float d = sm.v[pp][cl1_vidx<RPT>(st)];
    const float dd = fin ? d - mx : d;
    a.score[s] = dd > -INFINITY ? off + (double)dd : -INFINITY;
  }
  int thi = T - 1;
  while (thi > 0) {
    const int tlo = max(0, thi - TB);
    const int rows = thi - tlo;
    __syncthreads();
    for (int z = tid; z < rows * NP; z += NT) stage[z] = a.psi[(base + tlo + 1) * NP + z];
    __syncthreads();
    if (tid == 0) {
      for (int t = thi; t > tlo; --t) {
        a.path[base + t] = st;
        st = stage[(t - tlo - 1) * NP + st];
      }
    }
    thi = tlo;
  }
  if (tid == 0) a.path[base] = st;
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

template <int NP, int CLN>
cudaError_t launch_fb_cl1(const LargeArgs& a, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CLN, (unsigned)a.n_groups, 2);
  cfg.blockDim = dim3(Cl1<NP, CLN>::NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLN;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, large_fb_cl1_kernel<NP, CLN>, a);
}

bool large_cl1_supported(int NP, int group_fill) { return group_fill == 1 && (NP == 64 || NP == 128 || NP == 256); }

template <int NP, int CLN>
cudaError_t launch_vit_cl1(const LargeArgs& a, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CLN, (unsigned)a.n_groups, 1);
  cfg.blockDim = dim3(Cl1<NP, CLN>::NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CLN;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, large_vit_cl1_kernel<NP, CLN>, a);
}

cudaError_t launch_large_viterbi_cl1(int NP, const LargeArgs& a, cudaStream_t st) {
  switch (NP) {
    case 64: return launch_vit_cl1<64, 1>(a, st);
    case 128: return launch_vit_cl1<128, 2>(a, st);
    case 256: return launch_vit_cl1<256, 4>(a, st);
  }
  return cudaErrorInvalidValue;
}

// 64 columns per CTA: one CTA at padded N = 64, clusters of 2 and 4 above
cudaError_t launch_large_fb_cl1(int NP, const LargeArgs& a, cudaStream_t st) {
  switch (NP) {
    case 64: return launch_fb_cl1<64, 1>(a, st);
    case 128: return launch_fb_cl1<128, 2>(a, st);
    case 256: return launch_fb_cl1<256, 4>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hmm
