// Persistent-kernel families for cubic real grids n^3 (the real x stage works
// on n/2 complex pairs): R2C forward (x, y, z), C2R inverse (z, y, x), and
// the fused Poisson solve (x, y, fused z, y, x). Separate kernels per
// direction keep each one's register allocation to what it runs.
#include "gbfft_kernels.cuh"

namespace gbfft {

#define GBFFT_REAL_FAMILY(N)                                                                                   \
  v.push_back(make_persistent_entry<kcode(N / 2, kR2CPost, -1), kcode(N, kPlain, -1)>());                      \
  v.push_back(make_persistent_entry<kcode(N, kPlain, 1), kcode(N / 2, kC2RPre, 1)>());                         \
  v.push_back(make_persistent_entry<kcode(N / 2, kR2CPost, -1), kcode(N, kPlain, -1), kcode(N, kPoissonZ, -1), \
                                    kcode(N, kPlain, 1), kcode(N / 2, kC2RPre, 1)>());

void register_persistent_group_1(std::vector<PersistentKernel>& v) {
  GBFFT_REAL_FAMILY(64)
  GBFFT_REAL_FAMILY(128)
  GBFFT_REAL_FAMILY(256)
  GBFFT_REAL_FAMILY(512)
}

}  // namespace gbfft
