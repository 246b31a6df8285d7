// Shape selection and dispatch of the small-N fused E-step kernel.
#include "launch.h"

namespace hmm {

bool estep_small_supported(int NP, int G) {
  switch (NP) {
    case 2: return G == 1 || G == 2;
    case 4: return G == 1 || G == 2 || G == 4;
    case 8: return G == 2 || G == 4 || G == 8;
    case 16: return G == 4 || G == 8 || G == 16;
    case 32: return G == 16;
    default: return false;
  }
}

int default_estep_G(int NP, int64_t n_seq, int n_sm) {
  // Four states per lane measured fastest at N = 16 (fewest instructions
  // per state-step); wider chains only when the sequences would leave fewer
  // than about four warps per SM.
  if (NP == 32) return 16;
  int G = NP >= 4 ? NP / 4 : 1;
  if (!estep_small_supported(NP, G)) G = 1;
  while (G < 16 && G < NP && estep_small_supported(NP, 2 * G)) {
    const double warps = (double)n_seq / (16 / G);
    if (warps >= 4.0 * n_sm) break;
    G *= 2;
  }
  return G;
}

cudaError_t launch_estep_small(int NP, int G, int mode, const EStepArgs& a, int fam, int n_sm,
                               cudaStream_t st) {
  if (!estep_small_supported(NP, G)) return cudaErrorInvalidValue;
  switch (NP) {
    case 2:
    case 4: return launch_estep_np2_4(NP, G, mode, a, fam, n_sm, st);
    case 8: return launch_estep_np8(G, mode, a, fam, n_sm, st);
    case 16: return launch_estep_np16(G, mode, a, fam, n_sm, st);
    case 32: return launch_estep_np32(G, mode, a, fam, n_sm, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hmm
