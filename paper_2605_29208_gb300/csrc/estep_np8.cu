// E-step kernels for 8 (padded) states.
#include "estep_launch.cuh"

namespace hmm {
cudaError_t launch_estep_np8(int G, int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st) {
  if (G == 2) return estep_launch_modes<8, 2>(mode, a, fam, n_sm, st);
  if (G == 4) return estep_launch_modes<8, 4>(mode, a, fam, n_sm, st);
  if (G == 8) return estep_launch_modes<8, 8>(mode, a, fam, n_sm, st);
  return cudaErrorInvalidValue;
}
}  // namespace hmm
