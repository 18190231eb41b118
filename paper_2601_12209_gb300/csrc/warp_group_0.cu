// Warp-per-pencil stage kernels: complex lengths 512 and 256 (forward and
// inverse) and the real-data x stages of length 256 (R2C split, C2R merge).
#include "gbfft_warp.cuh"

namespace gbfft {

void register_warp_group_0(std::vector<WarpKernel>& v) {
  v.push_back(make_warp_entry<512, -1, kPlain>());
  v.push_back(make_warp_entry<512, 1, kPlain>());
  v.push_back(make_warp_entry<256, -1, kPlain>());
  v.push_back(make_warp_entry<256, 1, kPlain>());
  v.push_back(make_warp_entry<256, -1, kR2CPost>());
  v.push_back(make_warp_entry<256, 1, kC2RPre>());
}

}  // namespace gbfft
