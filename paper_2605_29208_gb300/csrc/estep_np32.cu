// E-step kernels for 32 (padded) states.
#include "estep_launch.cuh"

namespace hmm {
cudaError_t launch_estep_np32(int G, int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st) {
  if (G == 16) return estep_launch_modes<32, 16>(mode, a, fam, n_sm, st);
  return cudaErrorInvalidValue;
}
}  // namespace hmm
