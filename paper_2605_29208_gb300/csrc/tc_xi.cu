// xi on the tensor cores for large N (S6 of the path: sum_t xi_t as a GEMM
// with K = time):  Xi_c(i, j) = sum over the rows t < T-1 of chunk c's
// sequences of X_t(i) Y_t(j), with X_t = v_t / Z_t (forward row over Z_t) and
// Y_t = z_{t+1} = bt_{t+1} 2^(log2 b(t+1) - E_{t+1}).
//
// 1. xi_prep_kernel writes X and Y transposed (states x K, float32, K
//    contiguous) in a chunk-ordered K layout: the rows of a chunk's
//    sequences are consecutive, each chunk's range padded to a multiple of 32
//    with zeros; a 32 x 32 shared-memory transpose per block.
// 2. xi_tc_kernel: one CTA per (128 i, up to 256 j, chunk) tile; K-blocks of
//    32 (128 bytes) of X and Y move by TMA (2D tensor maps, 128-byte swizzle:
//    the K-major layout the MMA reads) into a ring of 4 stages with full /
//    empty mbarriers; one thread issues the copies, one thread issues
//    tcgen05.mma.kind::tf32 (M = 128, N = 256, K = 8) into TMEM; the
//    epilogue writes the float64 block.
// TF32 keeps float32's exponent range (1/Z_t can be large) with 10
// significant bits, the same as the FP16 recursions.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "launch.h"
#include "tc_common.cuh"

namespace hmm {
namespace {

using namespace tc;

constexpr int XI_KB = 32;          // K elements per block (128 bytes of TF32)
constexpr int XI_STAGES = 4;
constexpr int XI_TM = 128;

__global__ void __launch_bounds__(256) xi_prep_kernel(const float* __restrict__ fv, const float* __restrict__ bv,
                                                      const double* __restrict__ ob, const float* __restrict__ rz,
                                                      const float* __restrict__ logb, const int64_t* __restrict__ offsets,
                                                      const int32_t* __restrict__ tile_seq,
                                                      const int32_t* __restrict__ tile_row,
                                                      const int64_t* __restrict__ kseq, int NP, int N, int64_t ktot,
                                                      float* __restrict__ XT, float* __restrict__ YT) {
  __shared__ float xs[32][33], ysh[32][33];
  const int s = tile_seq[blockIdx.x];
  const int64_t b = offsets[s], e = offsets[s + 1];
  const int t0 = tile_row[blockIdx.x];
  const int i0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8
  // load: rows t0 + r (r = ty, ty + 8, ...), states i0 + tx
  for (int r = ty; r < 32; r += 8) {
    const int64_t t = b + t0 + r;
    float xv = 0.f, yv = 0.f;
    if (t + 1 < e) {
      const int i = i0 + tx;
      xv = fv[t * NP + i] * rz[t];
      if (i < N) {
        const float E = (float)(ob[t] - ob[t + 1]);
        const float w = bv[(t + 1) * NP + i];
        yv = w > 0.f ? exp2f(logb[(t + 1) * N + i] * 1.4426950408889634f + log2f(w) - E) : 0.f;
      }
    }
    xs[r][tx] = xv;
    ysh[r][tx] = yv;
  }
  __syncthreads();
  // store transposed: state i0 + r, K index kseq[s] + t0 + tx
  const int64_t k = kseq[s] + t0 + tx;
  const bool valid = b + t0 + tx + 1 < e;
  for (int r = ty; r < 32; r += 8) {
    if (valid) {
      XT[(size_t)(i0 + r) * ktot + k] = xs[tx][r];
      YT[(size_t)(i0 + r) * ktot + k] = ysh[tx][r];
    }
  }
}

// zeros in the padding of each chunk's K range: [kc0 + used, kc0 + padded)
__global__ void xi_pad_kernel(const int64_t* __restrict__ kc0, const int32_t* __restrict__ kused,
                              const int32_t* __restrict__ kpad, int NP, int64_t ktot, float* XT, float* YT) {
  const int c = blockIdx.x;
  const int npad = kpad[c] - kused[c];
  for (int z = threadIdx.x; z < npad * NP; z += blockDim.x) {
    const int i = z / npad, q = z % npad;
    const int64_t k = kc0[c] + kused[c] + q;
    XT[(size_t)i * ktot + k] = 0.f;
    YT[(size_t)i * ktot + k] = 0.f;
  }
}

// one 2D tensor-map tile (x = K element, y = state row) into shared memory,
// completing `bar`'s transaction count
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Stage ring: thread 0 loads K-block kb of the X tile (128 states) and the
// Y tile (TN states) with two TMA copies into stage kb % XI_STAGES once the
// MMAs of block kb - XI_STAGES have released it (`empty`); thread 32 issues
// the four MMAs of a block once its copies have landed (`full`) and releases
// the stage with tcgen05.commit.  The tensor maps' 128-byte swizzle is the
// K-major layout sw128_desc describes.
template <int TN>
__global__ void __launch_bounds__(128, 1) xi_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                       const __grid_constant__ CUtensorMap tmY,
                                                       const int64_t* __restrict__ kc0,
                                                       const int32_t* __restrict__ kpad, int NP,
                                                       double* __restrict__ xi_chunk, int* status) {
  constexpr uint32_t A_BYTES = XI_TM * 128, B_BYTES = TN * 128, STAGE = A_BYTES + B_BYTES;
  extern __shared__ uint8_t xr[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(xr) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + XI_STAGES * STAGE);   // [XI_STAGES] copies landed
  uint64_t* empty = full + XI_STAGES;                                     // [XI_STAGES] MMAs of the stage done
  uint64_t* done = empty + XI_STAGES;                                     // every MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tj_count = NP / TN;
  const int ti = blockIdx.x / tj_count, tj = blockIdx.x % tj_count;
  const int c = blockIdx.y;
  const int64_t k0 = kc0[c];
  const int nkb = kpad[c] / XI_KB;
  if (tid == 0) {
    for (int z = 0; z < XI_STAGES; ++z) {
      mbar_init(&full[z], 1);
      mbar_init(&empty[z], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmY)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % XI_STAGES;
      if (kb >= XI_STAGES && !mbar_wait(&empty[st], (uint32_t)((kb / XI_STAGES - 1) & 1)))
        set_status(status, ST_TIMEOUT);
      mbar_expect_tx(&full[st], STAGE);
      const uint32_t sa = smem_u32(sm + st * STAGE);
      const int x = (int)(k0 + (int64_t)kb * XI_KB);
      tma_load_2d(sa, &tmX, x, ti * XI_TM, smem_u32(&full[st]));
      tma_load_2d(sa + A_BYTES, &tmY, x, tj * TN, smem_u32(&full[st]));
    }
  } else if (tid == 32) {
    const uint32_t idesc = tc_idesc_tf32(XI_TM, TN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % XI_STAGES;
      if (!mbar_wait(&full[st], (uint32_t)((kb / XI_STAGES) & 1))) set_status(status, ST_TIMEOUT);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(sm + st * STAGE), sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = sw128_desc(sa + kk * 32), bd = sw128_desc(sb + kk * 32);
        const uint32_t acc = (kb | kk) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[st]))
                   : "memory");
    }
    if (nkb > 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(done))
                   : "memory");
  }
  __syncwarp();
  if (nkb > 0 && !mbar_wait(done, 0u))
    if ((tid & 31) == 0) set_status(status, ST_TIMEOUT);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: lane = row i of the tile, 32 columns per load
  double* out = xi_chunk + (size_t)c * NP * NP + (size_t)(ti * XI_TM + warp * 32 + (tid & 31)) * NP + tj * TN;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < TN; c0 += 32) {
    uint32_t r[32];
    if (nkb > 0) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(tl + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    } else {
#pragma unroll
      for (int z = 0; z < 32; ++z) r[z] = 0u;
    }
#pragma unroll
    for (int z = 0; z < 32; ++z) out[c0 + z] = (double)__uint_as_float(r[z]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// [rows][ktot] float32, K contiguous; box of 32 K elements (128 bytes) x box_rows
// states with 128-byte swizzle
cudaError_t make_xi_map(CUtensorMap* m, const float* base, int64_t ktot, int rows, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)ktot, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ktot * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)XI_KB, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int TN>
cudaError_t launch_xi_tn(const float* XT, const float* YT, int64_t ktot, const int64_t* kc0, const int32_t* kpad,
                         int n_chunks, int NP, double* xi_chunk, int* status, cudaStream_t st) {
  constexpr size_t smem = 1024 + (size_t)XI_STAGES * (XI_TM * 128 + TN * 128) + (2 * XI_STAGES + 1) * 8 + 16;
  // TMA coordinates are 32-bit; the K extent is a multiple of 32 (16-byte rows)
  if (ktot >= (int64_t(1) << 31) || ktot % XI_KB != 0) return cudaErrorInvalidValue;
  CUtensorMap mx, my;
  cudaError_t e = make_xi_map(&mx, XT, ktot, NP, XI_TM);
  if (e == cudaSuccess) e = make_xi_map(&my, YT, ktot, NP, TN);
  if (e != cudaSuccess) return e;
  auto kern = xi_tc_kernel<TN>;
  e = ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((NP / XI_TM) * (NP / TN)), (unsigned)n_chunks);
  kern<<<grid, 128, smem, st>>>(mx, my, kc0, kpad, NP, xi_chunk, status);
  return cudaGetLastError();
}

}  // namespace

bool tc_xi_supported(int NP) { return NP >= 128 && NP <= 1024; }

cudaError_t launch_tc_xi(const LargeArgs& a, const float* rz, const int32_t* tile_seq, const int32_t* tile_row,
                         int n_tiles, const int64_t* kseq, const int64_t* kc0, const int32_t* kused,
                         const int32_t* kpad, int n_chunks, int64_t ktot, float* XT, float* YT, double* xi_chunk,
                         int* status, cudaStream_t st) {
  const int NP = a.mv.NP, N = a.mv.N;
  if (n_chunks == 0) return cudaSuccess;
  if (n_tiles > 0) {
    xi_prep_kernel<<<dim3((unsigned)n_tiles, (unsigned)(NP / 32)), 256, 0, st>>>(
        a.fv, a.bv, a.ob, rz, a.logb, a.offsets, tile_seq, tile_row, kseq, NP, N, ktot, XT, YT);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  xi_pad_kernel<<<(unsigned)n_chunks, 256, 0, st>>>(kc0, kused, kpad, NP, ktot, XT, YT);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (NP >= 256) return launch_xi_tn<256>(XT, YT, ktot, kc0, kpad, n_chunks, NP, xi_chunk, status, st);
  return launch_xi_tn<128>(XT, YT, ktot, kc0, kpad, n_chunks, NP, xi_chunk, status, st);
}

}  // namespace hmm
