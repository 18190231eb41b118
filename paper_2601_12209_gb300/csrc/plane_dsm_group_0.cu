// Slab in-plane stage pairs of real transforms with the plane's intermediate in
// distributed shared memory: 512-point real rows, planes of ny = 512 and 256
// rows, forward (R2C x stage, then y) and inverse (y, then C2R x stage).
#include "gbfft_plane_dsm.cuh"

namespace gbfft {

void register_plane_dsm_group_0(std::vector<PlaneDsmKernel>& v) {
  v.push_back(make_plane_dsm_entry<512, -1>());
  v.push_back(make_plane_dsm_entry<512, 1>());
  v.push_back(make_plane_dsm_entry<256, -1>());
  v.push_back(make_plane_dsm_entry<256, 1>());
}

}  // namespace gbfft
