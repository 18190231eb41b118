// C2R x stages with cp.async prefetch of the next tile: half-spectrum lengths
// M = 128, 256, 512 (real rows of 256, 512, 1024 points).
#include "gbfft_prefetch.cuh"

namespace gbfft {

void register_prefetch_group_0(std::vector<PrefetchKernel>& v) {
  v.push_back(make_prefetch_entry<128>());
  v.push_back(make_prefetch_entry<256>());
  v.push_back(make_prefetch_entry<512>());
}

}  // namespace gbfft
