// Launch helper of the small-N E-step kernel (included by the per-NP
// translation units).
#pragma once

#include "launch.h"

namespace hmm {

template <int NP, int G, int MODE, int FAMK>
cudaError_t estep_launch_fam(const EStepArgs& a, int n_sm, cudaStream_t st) {
  constexpr int WPB = kWarpsPerBlock;
  const size_t smem = sizeof(WarpSmem<SmallCfg<NP, G>>) * WPB;
  auto kern = estep_small_kernel<NP, G, WPB, MODE, FAMK>;
  cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int want = (a.n_items + WPB - 1) / WPB;
  int grid = per_sm * n_sm;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  kern<<<grid, WPB * 32, smem, st>>>(a);
  return cudaGetLastError();
}

// fam: the batch's single emission family, FAM_TABLE or FAM_ANY (mixed)
template <int NP, int G, int MODE>
cudaError_t estep_launch_one(const EStepArgs& a, int fam, int n_sm, cudaStream_t st) {
  switch (fam) {
    case FAM_TABLE: return estep_launch_fam<NP, G, MODE, FAM_TABLE>(a, n_sm, st);
    case HMM_GAUSS: return estep_launch_fam<NP, G, MODE, HMM_GAUSS>(a, n_sm, st);
    case HMM_POISSON: return estep_launch_fam<NP, G, MODE, HMM_POISSON>(a, n_sm, st);
    case HMM_GAMMA: return estep_launch_fam<NP, G, MODE, HMM_GAMMA>(a, n_sm, st);
    case HMM_BETA: return estep_launch_fam<NP, G, MODE, HMM_BETA>(a, n_sm, st);
    case HMM_WEIBULL: return estep_launch_fam<NP, G, MODE, HMM_WEIBULL>(a, n_sm, st);
    case HMM_NEGBIN: return estep_launch_fam<NP, G, MODE, HMM_NEGBIN>(a, n_sm, st);
    case HMM_STUDENT_T: return estep_launch_fam<NP, G, MODE, HMM_STUDENT_T>(a, n_sm, st);
    case HMM_VONMISES: return estep_launch_fam<NP, G, MODE, HMM_VONMISES>(a, n_sm, st);
    default: return estep_launch_fam<NP, G, MODE, FAM_ANY>(a, n_sm, st);
  }
}

template <int NP, int G>
cudaError_t estep_launch_modes(int mode, const EStepArgs& a, int fam, int n_sm, cudaStream_t st) {
  switch (mode) {
    case MODE_GAMMA: return estep_launch_one<NP, G, MODE_GAMMA>(a, fam, n_sm, st);
    case MODE_STATS | MODE_GAMMA: return estep_launch_one<NP, G, MODE_STATS | MODE_GAMMA>(a, fam, n_sm, st);
    default: return estep_launch_one<NP, G, MODE_STATS>(a, fam, n_sm, st);
  }
}

}  // namespace hmm
