// Failure-detection self-test of the bounded device waits.
//
// The tensor-core kernels wait on mbarrier phases completed by copies and
// by the other CTAs of their cluster; every such wait gives up after a cycle
// limit, records ST_TIMEOUT in the context's sticky status word and lets the
// kernel run to its end, so a lost completion becomes an error status that
// the host reads (hmm_ctx_status) instead of a hung GPU.  This entry point
// exercises that path on purpose without any real failure: one thread
// initialises an mbarrier that nothing ever arrives on and waits for its
// first phase with the same bounded wait (tc::mbar_wait) and a caller-given
// limit.  It holds no tensor memory and starts no copy, so the kernel simply
// returns after the limit.
#include "launch.h"
#include "runtime.h"
#include "tc_common.cuh"

namespace hmm {
namespace {

__global__ void wait_selftest_kernel(long long limit, int* status, long long* waited) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const long long t0 = clock64();
  const bool done = tc::mbar_wait(&bar, 0, limit);   // nothing arrives: expires
  waited[0] = clock64() - t0;
  if (!done) set_status(status, ST_TIMEOUT);
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" hmm_status hmm_ctx_wait_selftest(hmm_ctx ctx, int64_t limit_cycles, int64_t* h_waited, void* stream) {
  try {
    HMM_REQUIRE(ctx != nullptr, "ctx is NULL");
    HMM_REQUIRE(limit_cycles >= 1 && limit_cycles <= (int64_t)tc::TC_WAIT_CYCLES,
                "limit_cycles must be in [1, the library's own wait limit]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the elapsed-cycle count lands in the context's first spare work counter
    long long* waited = reinterpret_cast<long long*>(ctx->counters + 32);
    wait_selftest_kernel<<<1, 32, 0, st>>>((long long)limit_cycles, ctx->status, waited);
    HMM_CUDA(cudaGetLastError());
    if (h_waited) {
      long long w = 0;
      HMM_CUDA(cudaMemcpyAsync(&w, waited, sizeof(w), cudaMemcpyDeviceToHost, st));
      HMM_CUDA(cudaStreamSynchronize(st));
      *h_waited = (int64_t)w;
    }
    return HMM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  }
}
