// Warp-per-pencil length-512 stage kernels, forward and inverse.
#include "gbfft_warp.cuh"

namespace gbfft {

void register_warp_group_0(std::vector<WarpKernel>& v) {
  v.push_back(make_warp_entry<-1>());
  v.push_back(make_warp_entry<1>());
}

}  // namespace gbfft
