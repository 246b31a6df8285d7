// Time-parallel forward-backward for long sequences at small N (padded N
// <= 32), used when a batch has too few sequences to fill the GPU with one
// chain per direction (the recursions are sequential in t).
//
// The forward step is v_t ~ v_{t-1} M_t with M_t = A diag(b_t), the backward
// step z_t ~ diag(b_t) A z_{t+1}.  A sequence is cut into chunks of L steps (chosen per plan):
//   1. tp_transfer_kernel: every chunk, in parallel, forms its transfer
//      matrix (product of its M_t, or of its diag(b_t) A), one warp per row,
//      each row scaled to a power-of-two exponent per step;
//   2. tp_boundary_kernel: one warp per sequence and direction walks the
//      chunks in order and applies the transfer matrices to the start vector:
//      the scaled forward (backward) vector at every chunk boundary;
//   3. tp_recompute_kernel: every chunk, in parallel, reruns its steps from
//      its boundary vector with exactly the per-step form of the large-N
//      recursion (v_t = 2^(log2 b + log2 s - E), float64 offsets) and writes
//      the same rows, so the posterior kernel of that path finishes the job.
// The result is the sequential recursion up to float32 rounding of the chunk
// products (the same matrices, associated differently).
//
// Every scale is a power of two with an integer exponent, so the exponents
// are carried in 64-bit integers: the sequential chains of all three kernels
// then run on the FP32 and integer pipes only (GB300's FP64 rate is a small
// fraction of its FP32 rate).  A single step's exponent (the floor of a row
// maximum of log2 densities) is taken to lie within +-2^31.  Exponents become
// float64 only where a row's offset is stored for the posterior kernel.
#include <climits>

#include "launch.h"

namespace hmm {
namespace {

constexpr float kL2e = 1.4426950408889634f;

__device__ __forceinline__ float wmax(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// lane `col` of a warp: log2 b_col(t) (-inf for padding or outside the support)
__device__ __forceinline__ float lb2_at(const float* logb, int64_t row, int N, int col) {
  return col < N ? __ldg(logb + row * N + col) * kL2e : -INFINITY;
}

// One warp per (chunk, direction, row r of the transfer matrix).  Lanes are
// the columns.  Forward: x <- (x A) .* b_t for t ascending; backward:
// x <- (x .* b_t) A for t ascending (row r of prod_t diag(b_t) A).  Each step
// the emissions are shifted by their row maximum and x by its own maximum;
// both exponents go into the row's float64 exponent.
template <int NP>
__global__ void __launch_bounds__(NP * 32) tp_transfer_kernel(TpArgs a) {
  const int c = blockIdx.x, dir = blockIdx.y;
  const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = a.chunk_seq[c];
  const int64_t base = a.offsets[s];
  const int T = (int)(a.offsets[s + 1] - base);
  const int t0 = a.chunk_t0[c], t1 = min(t0 + a.L, T);
  const int m = a.model_id[s];
  const int N = a.mv.N;
  // steps covered: forward skips t = 0 (the start vector), backward skips T-1
  const int lo = (dir == 0 && t0 == 0) ? 1 : t0;
  const int hi = (dir == 1 && t1 == T) ? T - 1 : t1;
  float Acol[NP];   // forward: column `lane` of A; backward: column `lane` as well (x A)
#pragma unroll
  for (int i = 0; i < NP; ++i) Acol[i] = lane < NP ? a.mv.A32[((size_t)m * NP + i) * NP + lane] : 0.f;
  float x = (lane == r) ? 1.f : 0.f;
  long long e = 0;
  for (int t = lo; t < hi; ++t) {
    const float lb = lb2_at(a.logb, base + t, N, lane);
    const float M = wmax(lb);
    const float Ms = M > -INFINITY ? floorf(M) : 0.f;
    const float b = exp2f(lb - Ms);
    e += (int)Ms;
    float y = 0.f;
    if (dir == 0) {
#pragma unroll
      for (int i = 0; i < NP; ++i) y = fmaf(__shfl_sync(0xffffffffu, x, i), Acol[i], y);
      y *= b;
    } else {
      const float xb = x * b;
#pragma unroll
      for (int i = 0; i < NP; ++i) y = fmaf(__shfl_sync(0xffffffffu, xb, i), Acol[i], y);
    }
    const float mx = wmax(y);
    const float E = mx > 0.f ? floorf(log2f(mx)) : 0.f;
    x = y * exp2f(-E);
    e += (int)E;
  }
  if (lane < NP) a.Q[(((size_t)c * 2 + dir) * NP + r) * NP + lane] = x;
  if (lane == 0) a.qexp[((size_t)c * 2 + dir) * NP + r] = e;
}

// One warp per (sequence, direction): the start vector, then the chunk
// transfers in order; the scaled vector after chunk c (forward: at its last
// step; backward: at its first step) goes to bvec[c][dir] with its offset.
template <int NP>
__global__ void tp_boundary_kernel(TpArgs a) {
  const int s = blockIdx.x, dir = blockIdx.y, lane = threadIdx.x;
  const int64_t base = a.offsets[s];
  const int T = (int)(a.offsets[s + 1] - base);
  if (T == 0) return;
  const int m = a.model_id[s];
  const int N = a.mv.N;
  const int c0 = a.seq_chunk0[s], nc = a.seq_nchunk[s];
  float w;
  long long O;
  {   // start: forward t = 0 (pi .* b_0), backward t = T-1 (b_{T-1})
    const float lb = lb2_at(a.logb, base + (dir == 0 ? 0 : T - 1), N, lane);
    const float u = dir == 0 ? lb + (lane < NP ? a.mv.logpi2[(size_t)m * NP + lane] : -INFINITY) : lb;
    const float mx = wmax(u);
    const float E = mx > -INFINITY ? floorf(mx) : 0.f;
    w = exp2f(u - E);
    O = (long long)E;
  }
  // the transfer data of chunk k + 1 are loaded while chunk k is applied
  // (the walk is sequential; this hides the load latency)
  float qv[NP], qn[NP];
  long long ev = 0, en = 0;
  auto load = [&](int k, float* q, long long& ex) {
    const int c = dir == 0 ? c0 + k : c0 + nc - 1 - k;
    const float* Q = a.Q + ((size_t)c * 2 + dir) * NP * NP;
    // forward: lane holds column `lane` (Q[r][lane], r < NP); backward: row `lane`
#pragma unroll
    for (int r = 0; r < NP; ++r) q[r] = lane < NP ? (dir == 0 ? Q[r * NP + lane] : Q[lane * NP + r]) : 0.f;
    ex = lane < NP ? a.qexp[((size_t)c * 2 + dir) * NP + lane] : 0;
  };
  if (nc > 0) load(0, qv, ev);
  for (int k = 0; k < nc; ++k) {
    const int c = dir == 0 ? c0 + k : c0 + nc - 1 - k;
    if (k + 1 < nc) load(k + 1, qn, en);
    // Lane r carries a value u_r 2^{ev_r} with u_r > 0 (forward: w_r times
    // row r of the chunk's matrix; backward: the dot of row r with w).  With
    // emax the largest ev_r among nonzero lanes, the lanes are brought to a
    // common exponent emax + G (G = floor of the largest log2 u_r + ev_r -
    // emax); exponent differences are clamped at -1000, far below float
    // underflow, so they stay small integers.
    float u;
    if (dir == 0) {
      u = w;
    } else {
      u = 0.f;
#pragma unroll
      for (int j = 0; j < NP; ++j) u = fmaf(qv[j], __shfl_sync(0xffffffffu, w, j), u);
    }
    const bool live = lane < NP && u > 0.f;
    long long em = live ? ev : LLONG_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long other = __shfl_xor_sync(0xffffffffu, em, o);
      em = other > em ? other : em;
    }
    const int di = live ? (int)max(ev - em, -1000LL) : 0;
    const float lu = live ? log2f(u) : -INFINITY;
    const float G = wmax(live ? lu + (float)di : -INFINITY);
    const int Gi = G > -INFINITY ? (int)floorf(G) : 0;
    const float f = live ? exp2f(lu + (float)(di - Gi)) : 0.f;
    float y;
    if (dir == 0) {
      // w Q = sum_r f_r Q'[r][:]
      y = 0.f;
#pragma unroll
      for (int r = 0; r < NP; ++r) y = fmaf(__shfl_sync(0xffffffffu, f, r), qv[r], y);
    } else {
      y = f;
    }
    if (em != LLONG_MIN) O += em + Gi;
    const float mx = wmax(y);
    const float E = mx > 0.f ? floorf(log2f(mx)) : 0.f;
    w = y * exp2f(-E);
    O += (int)E;
    if (lane < NP) a.bvec[((size_t)c * 2 + dir) * NP + lane] = w;
    if (lane == 0) a.boff[(size_t)c * 2 + dir] = O;
#pragma unroll
    for (int r = 0; r < NP; ++r) qv[r] = qn[r];
    ev = en;
  }
}

// One warp per (chunk, direction): rerun the chunk's steps from the boundary
// vector of the neighbouring chunk, writing the rows of the large-N path.
template <int NP>
__global__ void tp_recompute_kernel(TpArgs a) {
  const int c = blockIdx.x, dir = blockIdx.y, lane = threadIdx.x;
  const int s = a.chunk_seq[c];
  const int64_t base = a.offsets[s];
  const int T = (int)(a.offsets[s + 1] - base);
  const int t0 = a.chunk_t0[c], t1 = min(t0 + a.L, T);
  const int m = a.model_id[s];
  const int N = a.mv.N;
  const int c0 = a.seq_chunk0[s], nc = a.seq_nchunk[s];
  float Ar[NP];   // forward: column `lane` of A (s = v A); backward: row `lane` of A (s = A z)
#pragma unroll
  for (int i = 0; i < NP; ++i)
    Ar[i] = lane < NP ? (dir == 0 ? a.mv.A32[((size_t)m * NP + i) * NP + lane] : a.mv.A32[((size_t)m * NP + lane) * NP + i])
                      : 0.f;
  float v;
  long long O;
  int t, tend, step;
  if (dir == 0) {
    if (c == c0) {   // t = 0: pi .* b_0
      const float lb = lb2_at(a.logb, base, N, lane);
      const float u = lb + (lane < NP ? a.mv.logpi2[(size_t)m * NP + lane] : -INFINITY);
      const float mx = wmax(u);
      const float E = mx > -INFINITY ? floorf(mx) : 0.f;
      v = exp2f(u - E);
      O = (long long)E;
      if (lane < NP) a.fv[base * NP + lane] = v;
      if (lane == 0) a.oa[base] = (double)O;
      t = 1;
    } else {
      v = lane < NP ? a.bvec[((size_t)(c - 1) * 2 + 0) * NP + lane] : 0.f;
      O = a.boff[(size_t)(c - 1) * 2 + 0];
      t = t0;
    }
    tend = t1;
    step = 1;
  } else {
    if (c == c0 + nc - 1) {   // t = T-1: bt = 1, z = b_{T-1}
      const float lb = lb2_at(a.logb, base + T - 1, N, lane);
      const float mx = wmax(lb);
      const float E = mx > -INFINITY ? floorf(mx) : 0.f;
      if (lane < NP) a.bv[(base + T - 1) * NP + lane] = lane < N ? 1.f : 0.f;
      if (lane == 0) a.ob[base + T - 1] = 0.0;
      v = exp2f(lb - E);
      O = (long long)E;
      t = T - 2;
    } else {
      v = lane < NP ? a.bvec[((size_t)(c + 1) * 2 + 1) * NP + lane] : 0.f;
      O = a.boff[(size_t)(c + 1) * 2 + 1];
      t = t1 - 1;
    }
    tend = t0 - 1;
    step = -1;
  }
  for (; t != tend; t += step) {
    float sacc = 0.f;
#pragma unroll
    for (int i = 0; i < NP; ++i) sacc = fmaf(__shfl_sync(0xffffffffu, v, i), Ar[i], sacc);
    const int64_t row = base + t;
    if (dir == 1) {
      if (lane < NP) a.bv[row * NP + lane] = sacc;
      if (lane == 0) a.ob[row] = (double)O;
    }
    const float lb = lb2_at(a.logb, row, N, lane);
    const float u = lb + log2f(sacc);
    const float mx = wmax(lane < NP ? u : -INFINITY);
    const float E = mx > -INFINITY ? floorf(mx) : 0.f;
    v = exp2f(u - E);
    O += (int)E;
    if (dir == 0) {
      if (lane < NP) a.fv[row * NP + lane] = v;
      if (lane == 0) a.oa[row] = (double)O;
    }
  }
}

template <int NP>
cudaError_t launch_np(const TpArgs& a, int n_chunks, int n_seq, cudaStream_t st) {
  tp_transfer_kernel<NP><<<dim3((unsigned)n_chunks, 2), NP * 32, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tp_boundary_kernel<NP><<<dim3((unsigned)n_seq, 2), 32, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tp_recompute_kernel<NP><<<dim3((unsigned)n_chunks, 2), 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tp_fb(int NP, const TpArgs& a, int n_chunks, int n_seq, cudaStream_t st) {
  if (n_chunks == 0 || n_seq == 0) return cudaSuccess;
  switch (NP) {
    case 2: return launch_np<2>(a, n_chunks, n_seq, st);
    case 4: return launch_np<4>(a, n_chunks, n_seq, st);
    case 8: return launch_np<8>(a, n_chunks, n_seq, st);
    case 16: return launch_np<16>(a, n_chunks, n_seq, st);
    case 32: return launch_np<32>(a, n_chunks, n_seq, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hmm
