// E-step kernels for 16 (padded) states.
#include "estep_launch.cuh"

namespace hmm {
cudaError_t launch_estep_np16(int G, int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st) {
  if (G == 4) return estep_launch_modes<16, 4>(mode, a, fam, n_sm, st);
  if (G == 8) return estep_launch_modes<16, 8>(mode, a, fam, n_sm, st);
  if (G == 16) return estep_launch_modes<16, 16>(mode, a, fam, n_sm, st);
  return cudaErrorInvalidValue;
}
}  // namespace hmm
