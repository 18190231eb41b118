// Stage-kernel instantiations, group 2: lengths 96, 120, 128, 160.
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

void register_stage_group_2(std::vector<StageKernel>& v) {
  GBFFT_STAGE_COMPLEX(96)
  GBFFT_STAGE_REAL(96)
  GBFFT_STAGE_COMPLEX(120)
  GBFFT_STAGE_REAL(120)
  GBFFT_STAGE_COMPLEX(128)
  GBFFT_STAGE_REAL(128)
  GBFFT_STAGE_COMPLEX(160)
  GBFFT_STAGE_REAL(160)
}

}  // namespace gbfft
