// Launchers of the large-N kernels (padded N = 64 ... 1024).
#include "launch.h"
#include "mstep_types.h"

namespace hmm {

namespace {

// One warp per row: Z_t, gamma_t, 1/Z_t and (at t = 0) the log-likelihood.
// Block (sequence, slab): the slab's POST_SLAB rows of the sequence.
constexpr int64_t POST_SLAB = 2048;
__global__ void large_post_kernel(const float* __restrict__ fv, const float* __restrict__ bv,
                                  const double* __restrict__ oa, const double* __restrict__ ob,
                                  const int64_t* __restrict__ offsets, int NP, int N, float* __restrict__ gamma,
                                  float* __restrict__ rz, double* __restrict__ loglik, int* status) {
  const int s = blockIdx.x;
  const int64_t b = offsets[s], e = offsets[s + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (e == b) {
    if (threadIdx.x == 0 && blockIdx.y == 0 && loglik) loglik[s] = 0.0;
    return;
  }
  // rows of this block: slab blockIdx.y of POST_SLAB rows
  const int64_t r0 = b + (int64_t)blockIdx.y * POST_SLAB, r1 = min(e, r0 + POST_SLAB);
  for (int64_t t = r0 + warp; t < r1; t += nw) {
    float z = 0.f;
    for (int j = lane; j < NP; j += 32) z = fmaf(fv[t * NP + j], bv[t * NP + j], z);
    z = warp_sum_f(z);
    const float r = z > 0.f ? 1.f / z : 0.f;
    for (int j = lane; j < N; j += 32) gamma[t * N + j] = fv[t * NP + j] * bv[t * NP + j] * r;
    if (lane == 0) {
      rz[t] = r;
      if (t == b && loglik) {
        double ll = z > 0.f ? ((double)log2f(z) + oa[t] + ob[t]) * kLn2 : -INFINITY;
        if (!(z == z)) {
          ll = NAN;
          set_status(status, ST_NUMERIC);
        }
        loglik[s] = ll;
      }
    }
  }
}

// Per sequence and state: W, the family sums and gamma_1 (slot NST-1) from
// the occupancies; two-level float32 sums (64 steps in registers).
__global__ void large_stats_kernel(ModelView mv, const float* __restrict__ y, const float* __restrict__ gamma,
                                   const int64_t* __restrict__ offsets, const int32_t* __restrict__ model_id,
                                   bool table, float* __restrict__ part) {
  const int s = blockIdx.x;
  const int64_t b = offsets[s], e = offsets[s + 1];
  const int m = model_id[s];
  const int fam = mv.family[m];
  const int NP = mv.NP, N = mv.N;
  for (int j = threadIdx.x; j < NP; j += blockDim.x) {
    float st[NST], in[NST];
#pragma unroll
    for (int z = 0; z < NST; ++z) st[z] = in[z] = 0.f;
    if (j < N && e > b) {
      const float* c = mv.coef + ((size_t)m * NP + j) * KC;
      int cnt = 0;
      for (int64_t t = b; t < e; ++t) {
        const float g = gamma[t * N + j];
        if (g > 0.f) {
          in[0] += g;
          if (!table) {
            const Feat f = feat_of(fam, y[t], mv.lfact2);
            if (f.ok) accumulate_stats(fam, f, c, c + 4, g, in);
          }
        }
        if (++cnt == 64) {
#pragma unroll
          for (int z = 0; z < NST - 1; ++z) {
            st[z] += in[z];
            in[z] = 0.f;
          }
          cnt = 0;
        }
      }
#pragma unroll
      for (int z = 0; z < NST - 1; ++z) st[z] += in[z];
      st[NST - 1] = gamma[b * N + j];
    }
    float* out = part + ((size_t)s * NP + j) * NST;
#pragma unroll
    for (int z = 0; z < NST; ++z) out[z] = st[z];
  }
}

// Xi(i, j) = sum over a chunk's sequences and t < T-1 of v_t(i) y_t(j) with
// y_t(j) = z_{t+1}(j) / Z_t = 2^(log2 b_j(t+1) + log2 bt_{t+1}(j) - E_{t+1}) / Z_t,
// E_{t+1} = Ob_t - Ob_{t+1}.  64 x 64 output tile per block, 16 rows per
// shared-memory stage, float32 in registers flushed to float64 every 256 rows.
constexpr int XI_TILE = 64;
constexpr int XI_KT = 16;

__global__ void __launch_bounds__(256) large_xi_kernel(const float* __restrict__ fv, const float* __restrict__ bv,
                                                       const double* __restrict__ ob, const float* __restrict__ rz,
                                                       const float* __restrict__ logb, const int64_t* __restrict__ offsets,
                                                       const int32_t* __restrict__ seq_by_model,
                                                       const int32_t* __restrict__ chunk_lo,
                                                       const int32_t* __restrict__ chunk_hi, int NP, int N,
                                                       double* __restrict__ xi_chunk) {
  __shared__ __align__(16) float Xs[XI_KT][XI_TILE];
  __shared__ __align__(16) float Ys[XI_KT][XI_TILE];
  const int tiles = NP / XI_TILE;
  const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles;
  const int c = blockIdx.y;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  float acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f, dacc[p][q] = 0.0;
  int since = 0;
  for (int qs = chunk_lo[c]; qs < chunk_hi[c]; ++qs) {
    const int s = seq_by_model[qs];
    const int64_t b = offsets[s], e = offsets[s + 1];
    for (int64_t t0 = b; t0 + 1 < e; t0 += XI_KT) {
      for (int z = tid; z < XI_KT * XI_TILE; z += 256) {
        const int r = z / XI_TILE, col = z % XI_TILE;
        const int64_t t = t0 + r;
        float xv = 0.f, yv = 0.f;
        if (t + 1 < e) {
          const int i = ti * XI_TILE + col, j = tj * XI_TILE + col;
          xv = fv[t * NP + i];
          if (j < N) {
            const float E = (float)(ob[t] - ob[t + 1]);
            const float w = bv[(t + 1) * NP + j];
            yv = exp2f(logb[(t + 1) * N + j] * kLog2ef + log2f(w) - E) * rz[t];
          }
        }
        Xs[r][col] = xv;
        Ys[r][col] = yv;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < XI_KT; ++r) {
        const float4 x = *reinterpret_cast<const float4*>(&Xs[r][ty * 4]);
        const float4 yq = *reinterpret_cast<const float4*>(&Ys[r][tx * 4]);
        const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {yq.x, yq.y, yq.z, yq.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(xa[p], ya[q], acc[p][q]);
      }
      __syncthreads();
      since += XI_KT;
      if (since >= 256) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) dacc[p][q] += acc[p][q], acc[p][q] = 0.f;
        since = 0;
      }
    }
  }
  double* out = xi_chunk + (size_t)c * NP * NP;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = ti * XI_TILE + ty * 4 + p, j = tj * XI_TILE + tx * 4 + q;
      out[(size_t)i * NP + j] = dacc[p][q] + (double)acc[p][q];
    }
}

// Chunk records in the layout of rec_size(NP) from the per-sequence
// partials (fixed order) and the chunk's xi block.
__global__ void large_reduce_l1(const float* __restrict__ part, const double* __restrict__ loglik,
                                const double* __restrict__ xi_chunk, const int32_t* __restrict__ seq_by_model,
                                const int32_t* __restrict__ chunk_lo, const int32_t* __restrict__ chunk_hi, int NP,
                                double* __restrict__ chunk_rec) {
  const int c = blockIdx.x;
  const int lo = chunk_lo[c], hi = chunk_hi[c];
  const int RS = rec_size(NP);
  double* out = chunk_rec + (size_t)c * RS;
  // gridDim.y blocks share a chunk's fields (the xi block is a copy)
  for (int f = blockIdx.y * blockDim.x + threadIdx.x; f < RS; f += gridDim.y * blockDim.x) {
    double acc = 0.0;
    if (f == 0) {
      acc = (double)(hi - lo);
    } else if (f == 1) {
      for (int q = lo; q < hi; ++q) acc += loglik[seq_by_model[q]];
    } else if (f < rec_xi(NP)) {
      const int k = f - rec_g1(NP);
      for (int q = lo; q < hi; ++q) acc += (double)part[((size_t)seq_by_model[q] * NP + k) * NST + NST - 1];
    } else if (f < rec_st(NP)) {
      acc = xi_chunk[(size_t)c * NP * NP + (f - rec_xi(NP))];
    } else {
      const int k = (f - rec_st(NP)) / (NST - 1), z = (f - rec_st(NP)) % (NST - 1);
      for (int q = lo; q < hi; ++q) acc += (double)part[((size_t)seq_by_model[q] * NP + k) * NST + z];
    }
    out[f] = acc;
  }
}




template <int NP>
cudaError_t launch_fb_np(const LargeArgs& a, cudaStream_t st) {
  const size_t smem = LgShape<NP>::smem_bytes();
  auto kern = large_fb_kernel<NP>;
  cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)a.n_groups, 2), LG_NT, smem, st>>>(a);
  return cudaGetLastError();
}

// out[m][j][i] = ln a_ij (32 x 32 tiles through shared memory)
__global__ void logA_transpose_kernel(const float* __restrict__ in, int NP, float* __restrict__ out) {
  __shared__ float tile[32][33];
  const size_t off = (size_t)blockIdx.z * NP * NP;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) tile[r][threadIdx.x] = in[off + (size_t)(i0 + r) * NP + j0 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) out[off + (size_t)(j0 + r) * NP + i0 + threadIdx.x] = tile[threadIdx.x][r];
}

template <int NP>
cudaError_t launch_vit_np(const LargeArgs& a, cudaStream_t st) {
  const size_t smem = LgVitShape<NP>::smem_bytes();
  auto kern = large_viterbi_kernel<NP>;
  cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  logA_transpose_kernel<<<dim3(NP / 32, NP / 32, (unsigned)a.mv.M), dim3(32, 8), 0, st>>>(a.mv.logAe, NP, a.logAT);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)a.n_groups, LG_NT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_large_fb(int NP, const LargeArgs& a, cudaStream_t st) {
  if (a.n_groups == 0) return cudaSuccess;
  if (a.status && large_cl1_supported(NP, a.group_fill)) return launch_large_fb_cl1(NP, a, st);
  if (large_cl_supported(NP, a.n_groups)) return launch_large_fb_cl(a, st);
  switch (NP) {
    case 64: return launch_fb_np<64>(a, st);
    case 128: return launch_fb_np<128>(a, st);
    case 256: return launch_fb_np<256>(a, st);
    case 512: return launch_fb_np<512>(a, st);
    case 1024: return launch_fb_np<1024>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_large_post(const LargeArgs& a, int NP, int N, int64_t n_seq, int64_t max_T, float* gamma,
                              float* rz, double* loglik, int* status, cudaStream_t st) {
  if (n_seq == 0) return cudaSuccess;
  const unsigned slabs = (unsigned)std::max<int64_t>(1, (max_T + POST_SLAB - 1) / POST_SLAB);
  large_post_kernel<<<dim3((unsigned)n_seq, slabs), 256, 0, st>>>(a.fv, a.bv, a.oa, a.ob, a.offsets, NP, N, gamma, rz, loglik,
                                                     status);
  return cudaGetLastError();
}

cudaError_t launch_large_stats(const LargeArgs& a, const float* y, const float* gamma, int64_t n_seq, bool table,
                               float* part, cudaStream_t st) {
  if (n_seq == 0) return cudaSuccess;
  large_stats_kernel<<<(unsigned)n_seq, 256, 0, st>>>(a.mv, y, gamma, a.offsets, a.model_id, table, part);
  return cudaGetLastError();
}

cudaError_t launch_large_xi(const LargeArgs& a, const float* rz, const int32_t* seq_by_model, const int32_t* chunk_lo,
                            const int32_t* chunk_hi, int n_chunks, double* xi_chunk, cudaStream_t st) {
  if (n_chunks == 0) return cudaSuccess;
  const int tiles = a.mv.NP / XI_TILE;
  large_xi_kernel<<<dim3((unsigned)(tiles * tiles), (unsigned)n_chunks), 256, 0, st>>>(
      a.fv, a.bv, a.ob, rz, a.logb, a.offsets, seq_by_model, chunk_lo, chunk_hi, a.mv.NP, a.mv.N, xi_chunk);
  return cudaGetLastError();
}

cudaError_t launch_large_reduce(const float* part, const double* loglik, const double* xi_chunk,
                                const int32_t* seq_by_model, const int32_t* chunk_lo, const int32_t* chunk_hi,
                                int n_chunks, int NP, double* chunk_rec, cudaStream_t st) {
  if (n_chunks == 0) return cudaSuccess;
  const unsigned fy = (unsigned)std::min(std::max((rec_size(NP) + 255) / 256, 1), 1024);
  large_reduce_l1<<<dim3((unsigned)n_chunks, fy), 256, 0, st>>>(part, loglik, xi_chunk, seq_by_model, chunk_lo,
                                                                  chunk_hi, NP, chunk_rec);
  return cudaGetLastError();
}

cudaError_t launch_large_viterbi(int NP, const LargeArgs& a, cudaStream_t st) {
  if (a.n_groups == 0) return cudaSuccess;
  if (a.status && large_cl1_supported(NP, a.group_fill)) return launch_large_viterbi_cl1(NP, a, st);
  if (large_cl_supported(NP, a.n_groups)) return launch_large_viterbi_cl(a, st);
  switch (NP) {
    case 64: return launch_vit_np<64>(a, st);
    case 128: return launch_vit_np<128>(a, st);
    case 256: return launch_vit_np<256>(a, st);
    case 512: return launch_vit_np<512>(a, st);
    case 1024: return launch_vit_np<1024>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hmm
