// Instantiations and launcher of the small-N Viterbi kernel.
#include "launch.h"

namespace hmm {

namespace {

template <int NP, int G, int FAMK>
cudaError_t launch_fam(const VitArgs& a, int n_sm, cudaStream_t st) {
  constexpr int WPB = kWarpsPerBlock;
  const size_t smem = sizeof(VitSmem<VitCfg<NP, G>>) * WPB;
  auto kern = viterbi_small_kernel<NP, G, WPB, FAMK>;
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

template <int NP, int G>
cudaError_t launch_one(const VitArgs& a, int fam, int n_sm, cudaStream_t st) {
  switch (fam) {
    case FAM_TABLE: return launch_fam<NP, G, FAM_TABLE>(a, n_sm, st);
    case HMM_GAUSS: return launch_fam<NP, G, HMM_GAUSS>(a, n_sm, st);
    case HMM_POISSON: return launch_fam<NP, G, HMM_POISSON>(a, n_sm, st);
    case HMM_GAMMA: return launch_fam<NP, G, HMM_GAMMA>(a, n_sm, st);
    case HMM_BETA: return launch_fam<NP, G, HMM_BETA>(a, n_sm, st);
    case HMM_WEIBULL: return launch_fam<NP, G, HMM_WEIBULL>(a, n_sm, st);
    case HMM_NEGBIN: return launch_fam<NP, G, HMM_NEGBIN>(a, n_sm, st);
    case HMM_STUDENT_T: return launch_fam<NP, G, HMM_STUDENT_T>(a, n_sm, st);
    case HMM_VONMISES: return launch_fam<NP, G, HMM_VONMISES>(a, n_sm, st);
    default: return launch_fam<NP, G, FAM_ANY>(a, n_sm, st);
  }
}

}  // namespace

bool viterbi_small_supported(int NP, int G) {
  switch (NP) {
    case 2: return G == 1 || G == 2;
    case 4: return G == 1 || G == 2 || G == 4;
    case 8: return G == 2 || G == 4 || G == 8;
    case 16: return G == 4 || G == 8 || G == 16;
    case 32: return G == 16;
    default: return false;
  }
}

int default_viterbi_G(int NP, int64_t n_seq, int n_sm) {
  // Four states per lane unless the sequences would leave fewer than about
  // two warps per SM (measured on the N = 16 x 4096 workload).
  if (NP == 32) return 16;
  int G = NP >= 4 ? NP / 4 : 1;
  if (!viterbi_small_supported(NP, G)) G = 1;
  while (G < 16 && G < NP && viterbi_small_supported(NP, 2 * G)) {
    const double warps = (double)n_seq / viterbi_seqs_per_item(G);
    if (warps >= 2.0 * n_sm) break;
    G *= 2;
  }
  return G;
}

cudaError_t launch_viterbi_small(int NP, int G, const VitArgs& a, int fam, int n_sm,
                                 cudaStream_t st) {
#define HMM_CASE(np, g) \
  if (NP == np && G == g) return launch_one<np, g>(a, fam, n_sm, st);
  HMM_CASE(2, 1)
  HMM_CASE(2, 2)
  HMM_CASE(4, 1)
  HMM_CASE(4, 2)
  HMM_CASE(4, 4)
  HMM_CASE(8, 2)
  HMM_CASE(8, 4)
  HMM_CASE(8, 8)
  HMM_CASE(16, 4)
  HMM_CASE(16, 8)
  HMM_CASE(16, 16)
  HMM_CASE(32, 16)
#undef HMM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace hmm
