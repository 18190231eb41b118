// Warp-per-pencil stage kernels of length 1024 (32 values per lane: a radix-32
// step in registers, one transpose through the warp's region, radix 32 again),
// forward and inverse; any layout, and specialised for rows -> columns.
#include "gbfft_warp.cuh"

namespace gbfft {

void register_warp_group_1(std::vector<WarpKernel>& v) {
  v.push_back(make_warp_entry<1024, -1, kPlain>());
  v.push_back(make_warp_entry<1024, 1, kPlain>());
  v.push_back(make_warp_entry<1024, -1, kPlain, warp_io(kRow, kCol)>());
  v.push_back(make_warp_entry<1024, 1, kPlain, warp_io(kRow, kCol)>());
}

}  // namespace gbfft
