// Stage-kernel instantiations, group 7: lengths 960, 1024.
// Split across translation units so the library compiles in parallel.
#include "gbfft_kernels.cuh"

namespace gbfft {

#define GBFFT_STAGE_COMPLEX(L)                           \
  v.push_back(make_stage_entry<L, -1, kPlain>());        \
  v.push_back(make_stage_entry<L, 1, kPlain>());         \
  v.push_back(make_stage_entry<L, -1, kIdentity>());     \
  v.push_back(make_stage_entry<L, -1, kPoissonZ>());     \
  v.push_back(make_stage_entry<L, -1, kPoissonZB>());    \
  v.push_back(make_stage_entry<L, -1, kDct2>());         \
  v.push_back(make_stage_entry<L, 1, kDct3>());         \
  v.push_back(make_stage_entry<L, -1, kDst2>());         \
  v.push_back(make_stage_entry<L, 1, kDst3>());
#define GBFFT_STAGE_REAL(L)                              \
  v.push_back(make_stage_entry<L, -1, kR2CPost>());      \
  v.push_back(make_stage_entry<L, 1, kC2RPre>());

void register_stage_group_7(std::vector<StageKernel>& v) {
  GBFFT_STAGE_COMPLEX(960)
  GBFFT_STAGE_COMPLEX(1024)
}

}  // namespace gbfft
