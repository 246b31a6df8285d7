// k-means++ seeding and Lloyd iterations on the device for many restarts at
// once (the initialisation the paper names for Baum-Welch, Sec. 4.5; it
// gives no constants, the rules below are the library's reading).
//
// Features are float32 values; every distance, sum and centre is float64.
//   seeding: the first centre of restart r is observation floor(u_r0 T);
//     centre j is the first observation i whose running sum of D2(i) (the
//     squared distance to the nearest centre so far) exceeds u_rj times the
//     total (total 0: floor(u_rj T)).  One block per restart: each thread
//     owns a contiguous range of observations, the range sums are scanned in
//     a fixed order and the owning thread walks its range.
//   Lloyd: assignment to the nearest centre (the lowest index at ties), then
//     every non-empty cluster's centre moves to the mean of its observations;
//     a restart stops after the first pass that changes no assignment (or
//     after max_iter passes).  Cluster sums are block partials over fixed
//     ranges combined in a fixed order, so every result is bitwise
//     reproducible.
// The random numbers u are inputs (drawn by the caller), so a CPU reference
// can reproduce the seeding.
#include <algorithm>
#include <vector>

#include "launch.h"
#include "runtime.h"

namespace hmm {
namespace {

constexpr int KM_MAX_K = 64, KM_MAX_F = 16;
constexpr int KM_SEED_THREADS = 1024;
constexpr int KM_BLOCK = 256, KM_PPT = 8;   // points per thread of the assignment and sum kernels
constexpr int KM_PPB = KM_BLOCK * KM_PPT;

__device__ __forceinline__ double km_dist(const float* __restrict__ x, const double* __restrict__ c, int F) {
  double d = 0.0;
  for (int f = 0; f < F; ++f) {
    const double e = (double)x[f] - c[f];
    d = __dadd_rn(d, __dmul_rn(e, e));   // no contraction: the same rounding as a CPU sum of squares
  }
  return d;
}

// One block per restart: the K seeds (centres [R][K][F]; D2 scratch [R][T]).
__global__ void __launch_bounds__(KM_SEED_THREADS) km_seed_kernel(const float* __restrict__ X, int64_t T, int F,
                                                                  int K, const double* __restrict__ u,
                                                                  double* __restrict__ centres,
                                                                  double* __restrict__ d2all) {
  __shared__ double part[KM_SEED_THREADS];
  __shared__ double sh_pre, sh_target;
  __shared__ int sh_owner;
  __shared__ long long sel;
  const int r = blockIdx.x, tid = threadIdx.x;
  const double* ur = u + (size_t)r * K;
  double* C = centres + (size_t)r * K * F;
  double* d2 = d2all + (size_t)r * T;
  const int64_t L = (T + KM_SEED_THREADS - 1) / KM_SEED_THREADS;
  const int64_t lo = std::min<int64_t>(T, (int64_t)tid * L), hi = std::min<int64_t>(T, lo + L);
  for (int j = 0; j < K; ++j) {
    if (j == 0) {
      if (tid == 0) sel = std::min<int64_t>((int64_t)floor(ur[0] * (double)T), T - 1);
    } else {
      double s = 0.0;
      for (int64_t i = lo; i < hi; ++i) s += d2[i];
      part[tid] = s;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int q = 0; q < KM_SEED_THREADS; ++q) tot += part[q];
        sh_owner = -1;
        if (tot > 0.0) {
          const double target = ur[j] * tot;
          double pre = 0.0;
          int owner = KM_SEED_THREADS - 1;
          for (int q = 0; q < KM_SEED_THREADS; ++q) {
            if (pre + part[q] > target) {
              owner = q;
              break;
            }
            pre += part[q];
          }
          sh_pre = pre;
          sh_target = target;
          sh_owner = owner;
        } else {
          sel = std::min<int64_t>((int64_t)floor(ur[j] * (double)T), T - 1);
        }
      }
      __syncthreads();
      if (tid == sh_owner) {   // the first index of the range whose running sum passes the target
        double run = sh_pre;
        int64_t idx = hi > lo ? hi - 1 : T - 1;
        for (int64_t i = lo; i < hi; ++i) {
          run += d2[i];
          if (run > sh_target) {
            idx = i;
            break;
          }
        }
        sel = idx;
      }
    }
    __syncthreads();
    if (tid < F) C[(size_t)j * F + tid] = (double)X[sel * F + tid];
    __syncthreads();
    const double* cj = C + (size_t)j * F;
    for (int64_t i = lo; i < hi; ++i) {
      const double d = km_dist(X + i * F, cj, F);
      d2[i] = j == 0 ? d : fmin(d2[i], d);
    }
    __syncthreads();
  }
}

// Assignment pass: labels [R][T] of the nearest centre; changed[r] set when a
// label of restart r changes (every label counts as changed on pass 0).
__global__ void __launch_bounds__(KM_BLOCK) km_assign_kernel(const float* __restrict__ X, int64_t T, int F, int K,
                                                             const double* __restrict__ centres,
                                                             int32_t* __restrict__ labels, int pass,
                                                             int* __restrict__ changed,
                                                             const int* __restrict__ done) {
  __shared__ double Cs[KM_MAX_K * KM_MAX_F];
  const int r = blockIdx.y;
  if (done[r]) return;
  for (int z = threadIdx.x; z < K * F; z += blockDim.x) Cs[z] = centres[(size_t)r * K * F + z];
  __syncthreads();
  int ch = 0;
  int32_t* lab = labels + (size_t)r * T;
  for (int p = 0; p < KM_PPT; ++p) {
    const int64_t i = (int64_t)blockIdx.x * KM_PPB + (int64_t)p * KM_BLOCK + threadIdx.x;
    if (i >= T) break;
    double best = INFINITY;
    int bj = 0;
    for (int j = 0; j < K; ++j) {
      const double d = km_dist(X + i * F, Cs + j * F, F);
      if (d < best) {
        best = d;
        bj = j;
      }
    }
    if (pass == 0 || lab[i] != bj) ch = 1;
    lab[i] = bj;
  }
  if (__syncthreads_or(ch) && threadIdx.x == 0) atomicOr(&changed[r], 1);
}

// Per-block cluster sums [R][nb][K][F+1] (features, then the count) over the
// block's fixed range of observations, each a fixed-order tree reduction.
__global__ void __launch_bounds__(KM_BLOCK) km_sums_kernel(const float* __restrict__ X, int64_t T, int F, int K,
                                                           const int32_t* __restrict__ labels,
                                                           const int* __restrict__ done, double* __restrict__ part) {
  __shared__ double red[KM_BLOCK];
  const int r = blockIdx.y;
  if (done[r]) return;
  const int nb = gridDim.x;
  const int32_t* lab = labels + (size_t)r * T;
  int lj[KM_PPT];
  int64_t li[KM_PPT];
  for (int p = 0; p < KM_PPT; ++p) {
    const int64_t i = (int64_t)blockIdx.x * KM_PPB + (int64_t)p * KM_BLOCK + threadIdx.x;
    li[p] = i;
    lj[p] = i < T ? lab[i] : -1;
  }
  double* out = part + ((size_t)r * nb + blockIdx.x) * K * (F + 1);
  for (int j = 0; j < K; ++j)
    for (int f = 0; f <= F; ++f) {
      double v = 0.0;
      for (int p = 0; p < KM_PPT; ++p)
        if (lj[p] == j) v += f < F ? (double)X[li[p] * F + f] : 1.0;
      red[threadIdx.x] = v;
      __syncthreads();
      for (int w = KM_BLOCK / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
      }
      if (threadIdx.x == 0) out[j * (F + 1) + f] = red[0];
      __syncthreads();
    }
}

// Centres from the block sums (fixed order over blocks) when the pass changed
// an assignment; a restart whose pass changed nothing is done.
__global__ void km_update_kernel(int K, int F, int nb, const double* __restrict__ part, double* __restrict__ centres,
                                 int* __restrict__ changed, int* __restrict__ done, int* __restrict__ passes) {
  const int r = blockIdx.x;
  if (done[r]) return;
  const bool ch = changed[r] != 0;
  if (ch) {
    for (int z = threadIdx.x; z < K * F; z += blockDim.x) {
      const int j = z / F, f = z % F;
      double s = 0.0, n = 0.0;
      for (int b = 0; b < nb; ++b) {
        const double* pb = part + ((size_t)r * nb + b) * K * (F + 1) + j * (F + 1);
        s += pb[f];
        n += pb[F];
      }
      if (n > 0.0) centres[(size_t)r * K * F + z] = s / n;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    passes[r] += 1;
    if (!ch) done[r] = 1;
    changed[r] = 0;
  }
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" hmm_status hmm_kmeans(hmm_ctx ctx, const float* d_x, int64_t T, int32_t F, int32_t K, int32_t R,
                                 const double* h_u, int32_t max_iter, double* d_centres, int32_t* d_labels,
                                 int32_t* h_passes, void* stream) {
  try {
    HMM_REQUIRE(ctx && d_x && h_u && d_centres && d_labels, "NULL argument");
    HMM_REQUIRE(T >= 1 && T < (1ll << 40), "T must be in [1, 2^40)");
    HMM_REQUIRE(F >= 1 && F <= KM_MAX_F, "features per observation must be in [1, 16]");
    HMM_REQUIRE(K >= 1 && K <= KM_MAX_K, "clusters must be in [1, 64]");
    HMM_REQUIRE(R >= 1 && R <= 65535 && max_iter >= 0, "bad restart count or iteration limit");
    for (int64_t z = 0; z < (int64_t)R * K; ++z)
      HMM_REQUIRE(h_u[z] >= 0.0 && h_u[z] < 1.0, "the uniforms must lie in [0, 1)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nb = (int)((T + KM_PPB - 1) / KM_PPB);
    ctx->km_u.ensure((size_t)R * K * 8);
    ctx->km_d2.ensure((size_t)R * T * 8);
    ctx->km_part.ensure((size_t)R * nb * K * (F + 1) * 8);
    ctx->km_flags.ensure((size_t)R * 3 * 4);
    int* changed = ctx->km_flags.as<int>();
    int* done = changed + R;
    int* passes = done + R;
    HMM_CUDA(cudaMemcpyAsync(ctx->km_u.p, h_u, (size_t)R * K * 8, cudaMemcpyHostToDevice, st));
    HMM_CUDA(cudaMemsetAsync(changed, 0, (size_t)R * 3 * 4, st));
    km_seed_kernel<<<R, KM_SEED_THREADS, 0, st>>>(d_x, T, F, K, ctx->km_u.as<double>(), d_centres,
                                                  ctx->km_d2.as<double>());
    HMM_CUDA(cudaGetLastError());
    std::vector<int> hd((size_t)R);
    for (int it = 0; it < max_iter; ++it) {
      km_assign_kernel<<<dim3((unsigned)nb, (unsigned)R), KM_BLOCK, 0, st>>>(d_x, T, F, K, d_centres, d_labels, it,
                                                                             changed, done);
      km_sums_kernel<<<dim3((unsigned)nb, (unsigned)R), KM_BLOCK, 0, st>>>(d_x, T, F, K, d_labels, done,
                                                                           ctx->km_part.as<double>());
      km_update_kernel<<<R, 256, 0, st>>>(K, F, nb, ctx->km_part.as<double>(), d_centres, changed, done, passes);
      HMM_CUDA(cudaGetLastError());
      if ((it & 7) == 7 || it == max_iter - 1) {   // stop once every restart has converged
        HMM_CUDA(cudaMemcpyAsync(hd.data(), done, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
        HMM_CUDA(cudaStreamSynchronize(st));
        if (std::all_of(hd.begin(), hd.end(), [](int v) { return v != 0; })) break;
      }
    }
    if (h_passes) {
      HMM_CUDA(cudaMemcpyAsync(h_passes, passes, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
      HMM_CUDA(cudaStreamSynchronize(st));
    }
    return HMM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  }
}
