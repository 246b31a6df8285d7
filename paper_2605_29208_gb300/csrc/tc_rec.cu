// Tensor-core forward / backward recursions for large N (padded N = 64 ...
// 512): each step of Eq. 2 (and of the backward recursion) in the shifted
// exp-space form is a GEMM of the tile's 128 scaled vectors with A (or A^T),
// run by tcgen05.mma (FP16 operands, or TF32 for padded N <= 256; FP32
// accumulator in TMEM); the power-of-two row shift is added back in float64,
// as on the CUDA-core path.
//
// Work layout: a cluster of CL = NP / 64 CTAs owns a tile of 128 sequences
// of one model; CTA r computes the output states [64 r, 64 r + 64) of every
// step, so it keeps its 64 columns of A (FP16, per-column power-of-two scaled
// so that every column's maximum lies in [1, 2)) resident in shared memory,
// together with the full previous vector of the 128 sequences (FP16, the
// 128-byte-swizzled K-major layout the MMA reads).  Per step:
//   1. one thread issues 4 x CL MMAs (M = 128, N = 64, K = 16), K-block kb
//      as soon as its data have arrived (mbarrier per K-block);
//   2. every thread owns one sequence (one TMEM lane): it loads its 64
//      accumulators, forms u = log2 b + log2 s, and sends its partial row
//      maximum to every CTA of the cluster (st.async completing the
//      receiver's row-maximum mbarrier);
//   3. once the cluster's maxima are in, E = floor(max), v = 2^(u - E);
//      each warp writes its 32 rows of the FP16 slice into the CTA's own
//      K-block and pushes them to the other CTAs with 4 KB bulk copies that
//      complete their K-block barriers (no CTA-wide or cluster-wide barrier
//      inside the step).
// The rows written to global memory (forward v_t, backward bt_t = A z_{t+1},
// float64 offsets) have exactly the layout of the CUDA-core large-N kernel,
// so the posterior, statistics and xi kernels are shared.
//
// Every mbarrier wait is bounded; on expiry the kernel records ST_TIMEOUT
// and continues the protocol (so that all CTAs of a cluster still reach the
// same cluster barriers and the kernel ends), and TMEM is freed at the end.
#include <cuda_fp16.h>

#include "launch.h"
#include "tc_common.cuh"

namespace hmm {

namespace {

using namespace tc;

constexpr int TC_M = 128;        // sequences per tile (MMA M, TMEM lanes)
constexpr int TC_NC = 64;        // output states per CTA (MMA N, TMEM columns)
constexpr int TC_THREADS = 128;

struct TcArgs {
  const float* logb;         // [total_T][N] natural log
  const int64_t* offsets;
  const int32_t* model_id;
  const int32_t* tiles;      // [n_tiles][TC_M] sequence ids (one model per tile, first entry valid)
  int32_t n_tiles;
  ModelView mv;
  float* fv;
  float* bv;
  double* oa;
  double* ob;
  int* status;
};

// TF: TF32 operands (float32 rounded to 10 significant bits, float32's
// exponent range) instead of FP16; 32 K elements per 128-byte row, so a
// CTA's 64-state slice is two K-blocks.
template <int NP, bool TF>
struct TcShape {
  static constexpr int CL = NP / TC_NC;      // CTAs per cluster = state slices
  static constexpr int KPB = TF ? 32 : 64;   // K elements per 128-byte K-block row
  static constexpr int KBS = TC_NC / KPB;    // K-blocks per slice
  static constexpr uint32_t KB_V = TC_M * 128;          // one K-block of V
  static constexpr uint32_t SLICE_V = KB_V * KBS;       // one CTA's slice of V
  static constexpr uint32_t KB_B = TC_NC * 128;         // one K-block of B
  static constexpr uint32_t V_BYTES = (uint32_t)CL * SLICE_V;
  static constexpr uint32_t B_BYTES = (uint32_t)(NP / KPB) * KB_B;
  // at least 32 KB so that at most 7 CTAs (448 TMEM columns) share an SM
  static constexpr size_t smem_bytes() {
    const size_t b = 1024 + V_BYTES + B_BYTES + (size_t)CL * TC_M * 4 + 2 * 64 * 4 + (CL + 2) * 8 + 16;
    return b < 32768 ? 32768 : b;
  }
};

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
// Byte offset of element (row, k) in a [rows][32] TF32 K-block tile.
__device__ __forceinline__ uint32_t sw128_off32(int row, int k) {
  return sw128_chunk(row, k >> 2) + ((k & 3) << 2);
}

template <int NP, bool TF>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_fb_kernel(TcArgs a) {
  using S = TcShape<NP, TF>;
  constexpr int CL = S::CL;
  extern __shared__ uint8_t tc_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Vs = sm;
  uint8_t* Bs = Vs + S::V_BYTES;
  float* rmax = reinterpret_cast<float*>(Bs + S::B_BYTES);   // [CL][TC_M]
  float* csc = rmax + CL * TC_M;                             // [TC_NC] column scale exponents
  float* cinv = csc + TC_NC;                                 // [TC_NC] 2^-csc
  uint64_t* kbar = reinterpret_cast<uint64_t*>(cinv + TC_NC);// [CL] K-block data of the next MMA
  uint64_t* mbar = kbar + CL;                                // MMA completion
  uint64_t* rbar = mbar + 1;                                 // row maxima of the cluster
  uint32_t* tslot = reinterpret_cast<uint32_t*>(rbar + 1);
  __shared__ int s_tmax;

  const uint32_t rank = cluster_rank();
  const int tile = blockIdx.y, dir = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.mv.N;
  const int n0 = (int)rank * TC_NC;
  const int m = a.model_id[a.tiles[(size_t)tile * TC_M]];
  const int seq = a.tiles[(size_t)tile * TC_M + tid];
  int64_t base = 0;
  int len = 0;
  if (seq >= 0) {
    base = a.offsets[seq];
    len = (int)(a.offsets[seq + 1] - base);
  }
  if (tid == 0) {
    s_tmax = 0;
    // own K-block: one arrival per warp; the others: the local expect_tx
    for (int b = 0; b < CL; ++b) mbar_init(&kbar[b], b == (int)rank ? TC_THREADS / 32 : 1);
    mbar_init(mbar, 1);
    mbar_init(rbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_NC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  atomicMax(&s_tmax, len);
  // columns of A owned by this CTA: output state j = n0 + n reads
  //   forward  B(k, n) = a_kj (row j of A^T),  backward  B(k, n) = a_jk (row j of A)
  const float* src = (dir == 0 ? a.mv.AT32 : a.mv.A32) + (size_t)m * NP * NP;
  if (tid < TC_NC) {
    const float* row = src + (size_t)(n0 + tid) * NP;
    float mx = 0.f;
    for (int k = 0; k < NP; ++k) mx = fmaxf(mx, row[k]);
    csc[tid] = mx > 0.f ? -floorf(log2f(mx)) : 0.f;
    cinv[tid] = exp2f(-csc[tid]);
  }
  __syncthreads();
  for (int idx = tid; idx < TC_NC * NP; idx += TC_THREADS) {
    const int n = idx / NP, k = idx % NP;
    const float v = src[(size_t)(n0 + n) * NP + k] * exp2f(csc[n]);
    if constexpr (TF)
      *reinterpret_cast<uint32_t*>(Bs + (k >> 5) * S::KB_B + sw128_off32(n, k & 31)) = to_tf32(v);
    else
      *reinterpret_cast<__half*>(Bs + (k >> 6) * S::KB_B + sw128_off(n, k & 63)) = __float2half_rn(v);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int tmax = s_tmax;
  cluster_sync();   // every CTA's barriers are initialised before any copy targets them

  const bool vec = (n0 + TC_NC <= N) && (N % 4 == 0);
  float w[TC_NC];   // ln b of the step (loaded a step ahead), then u = log2 b + log2 s
  auto load_lb = [&](int k) {
    const bool act = k < len;
    const int64_t grow = base + (dir == 0 ? k : len - 1 - k);
    const float* p = a.logb + grow * N + n0;
    if (act && vec) {
#pragma unroll
      for (int c = 0; c < TC_NC; c += 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p + c));
        w[c] = q.x;
        w[c + 1] = q.y;
        w[c + 2] = q.z;
        w[c + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < TC_NC; ++c) w[c] = (act && n0 + c < N) ? __ldg(p + c) : -INFINITY;
    }
  };
  load_lb(0);
  double O = 0.0;
  const uint32_t idesc = TF ? tc_idesc_tf32(TC_M, TC_NC) : tc_idesc(TC_M, TC_NC);
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);

  for (int k = 0; k < tmax; ++k) {
    const bool act = k < len;
    const int64_t grow = base + (dir == 0 ? k : len - 1 - k);
    if (tid == 0) mbar_expect_tx(rbar, (uint32_t)(CL * TC_M * 4));
    if (k > 0) {
      if (tid == 0) {
        for (int kb = 0; kb < CL; ++kb) {
          if (!mbar_wait(&kbar[kb], (uint32_t)((k - 1) & 1))) set_status(a.status, ST_TIMEOUT);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int sb = 0; sb < S::KBS; ++sb) {
            const uint32_t va = smem_u32(Vs + kb * S::SLICE_V + sb * S::KB_V);
            const uint32_t ba = smem_u32(Bs + (kb * S::KBS + sb) * S::KB_B);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sw128_desc(va + kk * 32), bd = sw128_desc(ba + kk * 32);
              const uint32_t acc = (kb | sb | kk) ? 1u : 0u;
              if constexpr (TF)
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
              else
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(mbar))
                     : "memory");
      }
      __syncwarp();
      if (!mbar_wait(mbar, (uint32_t)((k - 1) & 1))) set_status(a.status, ST_TIMEOUT);
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tl + 32 * h));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float* q = a.bv + grow * NP + n0 + 32 * h;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          float sv[4];
#pragma unroll
          for (int z = 0; z < 4; ++z) {
            const int cc = 32 * h + c + z;
            const float sc = __uint_as_float(r[c + z]);
            sv[z] = sc * cinv[cc];
            w[cc] = fmaf(w[cc], kLog2ef, lg2a(sc) - csc[cc]);   // w: ln b -> u
          }
          if (dir == 1 && act) *reinterpret_cast<float4*>(q + c) = make_float4(sv[0], sv[1], sv[2], sv[3]);
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < TC_NC; ++c)
        w[c] = w[c] * kLog2ef + (dir == 0 ? a.mv.logpi2[(size_t)m * NP + n0 + c] : 0.f);
      if (dir == 1 && act) {
        float* q = a.bv + grow * NP + n0;
#pragma unroll
        for (int c = 0; c < TC_NC; ++c) q[c] = (n0 + c < N) ? 1.f : 0.f;
      }
    }
    // partial row maximum to every CTA of the cluster
    float mx = -INFINITY;
#pragma unroll
    for (int c = 0; c < TC_NC; ++c) mx = fmaxf(mx, w[c]);
    const uint32_t raddr = smem_u32(rmax + rank * TC_M + tid), rb = smem_u32(rbar);
#pragma unroll
    for (int p = 0; p < CL; ++p)
      asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(
                       mapa(raddr, (uint32_t)p)),
                   "f"(mx), "r"(mapa(rb, (uint32_t)p))
                   : "memory");
    if (!mbar_wait(rbar, (uint32_t)(k & 1))) set_status(a.status, ST_TIMEOUT);
    float M = -INFINITY;
#pragma unroll
    for (int p = 0; p < CL; ++p) M = fmaxf(M, rmax[p * TC_M + tid]);
    const float E = M > -INFINITY ? floorf(M) : 0.f;
    if (dir == 1 && rank == 0 && act) a.ob[grow] = O;
    O = (k == 0 ? 0.0 : O) + (double)E;
    if (dir == 0 && rank == 0 && act) a.oa[grow] = O;
    // new vector: float32 rows to global, the FP16 / TF32 slice into slice `rank`
    uint8_t* vrow = Vs + rank * S::SLICE_V;
#pragma unroll
    for (int c = 0; c < TC_NC; c += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = ex2f(w[c + q] - E);
      if (dir == 0 && act) {
        float* g = a.fv + grow * NP + n0 + c;
        *reinterpret_cast<float4*>(g) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(g + 4) = make_float4(v[4], v[5], v[6], v[7]);
      }
      if constexpr (TF) {
        uint8_t* blk = vrow + (c >> 5) * S::KB_V;
        const int q0 = (c & 31) >> 2;
        *reinterpret_cast<uint4*>(blk + sw128_chunk(tid, q0)) =
            make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
        *reinterpret_cast<uint4*>(blk + sw128_chunk(tid, q0 + 1)) =
            make_uint4(to_tf32(v[4]), to_tf32(v[5]), to_tf32(v[6]), to_tf32(v[7]));
      } else {
        __half2 h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
        *reinterpret_cast<uint4*>(vrow + sw128_off(tid, c)) = *reinterpret_cast<uint4*>(h);
      }
    }
    // this warp's 32 rows of the slice (4 KB, contiguous in the swizzled
    // layout) go to the other CTAs; the local K-block counts one arrival per warp
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (k + 1 < tmax && (tid & 31) == 0) {
      for (int p = 0; p < CL; ++p) {
        if (p == (int)rank) continue;
        const uint32_t bar = mapa(smem_u32(&kbar[rank]), (uint32_t)p);
        for (int sb = 0; sb < S::KBS; ++sb) {
          const uint32_t srcv = smem_u32(vrow + sb * S::KB_V + warp * 4096);
          asm volatile(
              "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  mapa(srcv, (uint32_t)p)),
              "r"(srcv), "r"(4096), "r"(bar)
              : "memory");
        }
      }
      mbar_arrive(&kbar[rank]);
      if (tid == 0)
        for (int kb = 0; kb < CL; ++kb)
          if (kb != (int)rank) mbar_expect_tx(&kbar[kb], S::SLICE_V);
    }
    if (k + 1 < tmax) load_lb(k + 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NC));
}

template <int NP, bool TF>
cudaError_t launch_tc_np(const TcArgs& a, cudaStream_t st) {
  using S = TcShape<NP, TF>;
  auto kern = tc_fb_kernel<NP, TF>;
  {
    cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), S::smem_bytes());
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S::CL, (unsigned)a.n_tiles, 2);
  cfg.blockDim = dim3(TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = S::smem_bytes();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

int tc_tile_rows() { return TC_M; }

bool tc_supported(int NP) { return NP >= 64 && NP <= 512; }

// the TF32 vector of a 128-sequence tile is 512 B per sequence at N = 512:
// with A's columns it no longer fits in shared memory
bool tc_tf32_supported(int NP) { return NP >= 64 && NP <= 256; }

cudaError_t launch_tc_fb(int NP, const LargeArgs& la, const int32_t* tiles, int n_tiles, int* status, bool tf32,
                         cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  TcArgs a;
  a.logb = la.logb;
  a.offsets = la.offsets;
  a.model_id = la.model_id;
  a.tiles = tiles;
  a.n_tiles = n_tiles;
  a.mv = la.mv;
  a.fv = la.fv;
  a.bv = la.bv;
  a.oa = la.oa;
  a.ob = la.ob;
  a.status = status;
  if (tf32) {
    switch (NP) {
      case 64: return launch_tc_np<64, true>(a, st);
      case 128: return launch_tc_np<128, true>(a, st);
      case 256: return launch_tc_np<256, true>(a, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (NP) {
    case 64: return launch_tc_np<64, false>(a, st);
    case 128: return launch_tc_np<128, false>(a, st);
    case 256: return launch_tc_np<256, false>(a, st);
    case 512: return launch_tc_np<512, false>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hmm
