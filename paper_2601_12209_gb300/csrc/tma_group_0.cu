// TMA stage-kernel instantiations, group 0: lengths 64, 128, 256.
#include "gbfft_kernels.cuh"
#include "gbfft_tma.cuh"

namespace gbfft {

template <int L, int DIR, int KIND, int SRC>
static TmaKernel tma_entry() {
  return TmaKernel{L, DIR, KIND, SRC, reinterpret_cast<const void*>(&tma_stage_kernel<L, DIR, KIND, SRC>),
                   tma_threads(L), TmaGeom<L, KIND, SRC>::smem};
}

#define GBFFT_TMA_COMPLEX(L)                                  \
  v.push_back(tma_entry<L, -1, kPlain, kTmaRow>());           \
  v.push_back(tma_entry<L, -1, kPlain, kTmaCol>());           \
  v.push_back(tma_entry<L, 1, kPlain, kTmaRow>());            \
  v.push_back(tma_entry<L, 1, kPlain, kTmaCol>());            \
  v.push_back(tma_entry<L, -1, kPoissonZ, kTmaRow>());        \
  v.push_back(tma_entry<L, -1, kPoissonZ, kTmaCol>());
#define GBFFT_TMA_REAL(L)                                     \
  v.push_back(tma_entry<L, -1, kR2CPost, kTmaRow>());         \
  v.push_back(tma_entry<L, 1, kC2RPre, kTmaCol>());

void register_tma_group_0(std::vector<TmaKernel>& v) {
  GBFFT_TMA_COMPLEX(64)
  GBFFT_TMA_REAL(64)
  GBFFT_TMA_COMPLEX(128)
  GBFFT_TMA_REAL(128)
  GBFFT_TMA_COMPLEX(256)
  GBFFT_TMA_REAL(256)
}

}  // namespace gbfft
