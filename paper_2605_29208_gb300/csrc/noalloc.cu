// hmm_forward_backward_static: forward-backward that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they want a
// posterior: code running inside a memory pool that forbids outside
// allocations, a real-time loop where cudaMalloc's implicit device
// synchronisation and unbounded latency are not acceptable, or a host that
// has reserved all free memory for itself.  This entry point serves them.
// It runs the same fused E-step kernel as hmm_forward_backward, but its
// scratch (the recurrence rows, the processing order and the work counter)
// lives in one file-scope __device__ array of fixed size, so the call issues
// no cudaMalloc, cudaFree or allocating library routine.  The caller still
// provides the batch, the model and the output buffers.
//
// The array is a global of the library: every GPU that loads the library
// holds kStaticScratchBytes of device memory until the process exits, all
// calls share it and it keeps the contents of the last call.  The parts that
// must start at zero are cleared on the stream by every call.  Two calls
// whose work overlaps on the GPU (different streams without ordering, or
// different host threads) race on the array and give undefined results.
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress); make that first call before any stream capture.
//
// The batch arrays live on the device, and reading them back to check them
// would need a synchronising copy, which is what these callers cannot take.
// So a small kernel checks them on the device before the E-step: offsets[0]
// = 0, non-decreasing offsets, offsets[n_seq] = total_T and model ids inside
// [0, n_models).  A malformed batch runs no sequence at all (the E-step's
// work counter starts past its last work item, so nothing reads or writes
// outside the caller's buffers or the scratch), every d_loglik entry is set
// to NaN and the model context's sticky status records HMM_E_ARG
// (hmm_ctx_status).  The call restores the caller's current device.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "launch.h"
#include "runtime.h"

namespace hmm {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 128;
void* g_static_addr[kMaxDevices] = {nullptr};
std::mutex g_static_mu;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// flags[0] != 0 after this kernel when the batch is malformed
__global__ void validate_batch_kernel(const int64_t* offsets, const int32_t* model_id, int64_t n_seq,
                                      int64_t total_T, int n_models, int* flags) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= n_seq;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = offsets[s];
    bool ok = s == 0 ? o == 0 : o >= offsets[s - 1];
    if (s == n_seq) ok = ok && o == total_T;
    else ok = ok && model_id[s] >= 0 && model_id[s] < n_models;
    if (!ok) atomicOr(flags, 1);
  }
}

// processing order = input order; on a malformed batch: no work items, NaN
// log-likelihoods and the ST_ARG status bit
__global__ void static_prepare_kernel(int32_t* order, int64_t n, const int* flags, int* work_counter,
                                      int n_items, double* loglik, int* status) {
  const bool bad = *flags != 0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    order[i] = (int32_t)i;
    if (bad) loglik[i] = nan("");
  }
  if (bad && i == 0) {
    *work_counter = n_items;
    set_status(status, ST_ARG);
  }
}

// Makes `device` current for the lifetime of the guard and then restores
// the caller's device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int device) {
    HMM_CUDA(cudaGetDevice(&prev));
    if (prev != device) HMM_CUDA(cudaSetDevice(device));
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Device address of the static array on the current device (looked up once
// per device; in host code the array's name is only a host-side handle).
void* static_scratch_address(int device) {
  HMM_REQUIRE(device >= 0 && device < kMaxDevices, "device index out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[device]) {
    void* p = nullptr;
    HMM_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[device] = p;
  }
  return g_static_addr[device];
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" hmm_status hmm_forward_backward_static(hmm_model model, const hmm_batch* batch,
                                                  const float* d_logb, float* d_gamma,
                                                  double* d_loglik, void* stream) {
  try {
    HMM_REQUIRE(model && batch && d_gamma && d_loglik, "NULL argument");
    HMM_REQUIRE(batch->n_seq >= 0 && batch->total_T >= 0, "negative batch sizes");
    HMM_REQUIRE(batch->n_seq < (1ll << 31) && batch->total_T < (1ll << 40), "batch too large");
    HMM_REQUIRE(batch->offsets != nullptr && (batch->n_seq == 0 || batch->model_id != nullptr),
                "batch arrays are NULL");
    HMM_REQUIRE(batch->total_T == 0 || batch->values != nullptr || d_logb != nullptr,
                "batch values are NULL");
    HMM_REQUIRE(batch->dim == model->D, "batch dim does not match the model");
    if (model->NP > 32) throw Error{HMM_E_UNSUPPORTED, "state counts above 32 are not supported"};
    if (model->table_family() && !d_logb)
      throw Error{HMM_E_UNSUPPORTED, "multivariate families need an emission table (d_logb)"};
    const int NP = model->NP;
    const int64_t S = batch->n_seq;
    // scratch layout: [0] work counter, [1] malformed-batch flag, the order
    // at byte 256, the recurrence rows after it
    const size_t order_off = 256;
    const size_t rows_off = order_off + align256((size_t)S * 4);
    const size_t need = rows_off + (size_t)batch->total_T * NP * 4;
    if (need > kStaticScratchBytes)
      throw Error{HMM_E_ARG, "batch needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                                 std::to_string(kStaticScratchBytes) + " (total_T * padded states * 4 + n_seq * 4 + 512)"};
    DeviceGuard dg(model->ctx->device);
    unsigned char* base = static_cast<unsigned char*>(static_scratch_address(model->ctx->device));
    if (S == 0) return HMM_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int* counter = reinterpret_cast<int*>(base);
    int* flags = counter + 1;
    int32_t* order = reinterpret_cast<int32_t*>(base + order_off);
    float* rows = reinterpret_cast<float*>(base + rows_off);
    const int G = default_estep_G(NP, S, model->ctx->n_sm);
    const int n_items = (int)((S + estep_seqs_per_item(G) - 1) / estep_seqs_per_item(G));
    HMM_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
    const unsigned vgrid = (unsigned)std::min<int64_t>((S + 256) / 256, 4 * (int64_t)model->ctx->n_sm);
    validate_batch_kernel<<<vgrid, 256, 0, st>>>(batch->offsets, batch->model_id, S, batch->total_T, model->M,
                                                 flags);
    HMM_CUDA(cudaGetLastError());
    static_prepare_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(order, S, flags, counter, n_items, d_loglik,
                                                                       model->ctx->status);
    HMM_CUDA(cudaGetLastError());
    EStepArgs a;
    a.y = batch->values;
    a.logb = d_logb;
    a.offsets = batch->offsets;
    a.model_id = batch->model_id;
    a.order = order;
    a.n_seq = (int32_t)S;
    a.n_items = n_items;
    a.mv = model->view();
    a.scratch = rows;
    a.gamma = d_gamma;
    a.partials = nullptr;   // no statistics in this mode
    a.loglik = d_loglik;
    a.work_counter = counter;
    a.status = model->ctx->status;
    int fam = model->h_family[0];
    for (int f : model->h_family)
      if (f != fam) fam = FAM_ANY;
    if (d_logb) fam = FAM_TABLE;
    HMM_CUDA(launch_estep_small(NP, G, MODE_GAMMA, a, fam, model->ctx->n_sm, st));
    return HMM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return HMM_E_ARG;
  }
}
