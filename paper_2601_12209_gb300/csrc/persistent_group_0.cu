// Persistent-kernel families for cubic complex-to-complex grids: one kernel
// per length and direction (forward: x, y, z stages; inverse: z, y, x).
#include "gbfft_kernels.cuh"

namespace gbfft {

#define GBFFT_C2C_FAMILY(L)                                             \
  v.push_back(make_persistent_entry<kcode(L, kPlain, -1)>());           \
  v.push_back(make_persistent_entry<kcode(L, kPlain, 1)>());

void register_persistent_group_0(std::vector<PersistentKernel>& v) {
  GBFFT_C2C_FAMILY(64)
  GBFFT_C2C_FAMILY(128)
  GBFFT_C2C_FAMILY(256)
  GBFFT_C2C_FAMILY(512)
  GBFFT_C2C_FAMILY(1024)
}

}  // namespace gbfft
