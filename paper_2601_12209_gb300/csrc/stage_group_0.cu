// Stage-kernel instantiations, group 0: lengths 2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 20, 24, 30, 32.
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

void register_stage_group_0(std::vector<StageKernel>& v) {
  GBFFT_STAGE_COMPLEX(2)
  GBFFT_STAGE_REAL(2)
  GBFFT_STAGE_COMPLEX(3)
  GBFFT_STAGE_REAL(3)
  GBFFT_STAGE_COMPLEX(4)
  GBFFT_STAGE_REAL(4)
  GBFFT_STAGE_COMPLEX(5)
  GBFFT_STAGE_REAL(5)
  GBFFT_STAGE_COMPLEX(6)
  GBFFT_STAGE_REAL(6)
  GBFFT_STAGE_COMPLEX(8)
  GBFFT_STAGE_REAL(8)
  GBFFT_STAGE_COMPLEX(10)
  GBFFT_STAGE_REAL(10)
  GBFFT_STAGE_COMPLEX(12)
  GBFFT_STAGE_REAL(12)
  GBFFT_STAGE_COMPLEX(15)
  GBFFT_STAGE_REAL(15)
  GBFFT_STAGE_COMPLEX(16)
  GBFFT_STAGE_REAL(16)
  GBFFT_STAGE_COMPLEX(20)
  GBFFT_STAGE_REAL(20)
  GBFFT_STAGE_COMPLEX(24)
  GBFFT_STAGE_REAL(24)
  GBFFT_STAGE_COMPLEX(30)
  GBFFT_STAGE_REAL(30)
  GBFFT_STAGE_COMPLEX(32)
  GBFFT_STAGE_REAL(32)
}

}  // namespace gbfft
