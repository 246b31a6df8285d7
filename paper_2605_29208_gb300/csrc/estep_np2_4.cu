// E-step kernels for 2 and 4 (padded) states.
#include "estep_launch.cuh"

namespace hmm {
cudaError_t launch_estep_np2_4(int NP, int G, int mode, const EStepArgs& a, int fam, int n_sm,
                               cudaStream_t st) {
  if (NP == 2 && G == 1) return estep_launch_modes<2, 1>(mode, a, fam, n_sm, st);
  if (NP == 2 && G == 2) return estep_launch_modes<2, 2>(mode, a, fam, n_sm, st);
  if (NP == 4 && G == 1) return estep_launch_modes<4, 1>(mode, a, fam, n_sm, st);
  if (NP == 4 && G == 2) return estep_launch_modes<4, 2>(mode, a, fam, n_sm, st);
  if (NP == 4 && G == 4) return estep_launch_modes<4, 4>(mode, a, fam, n_sm, st);
  return cudaErrorInvalidValue;
}
}  // namespace hmm
