// Fused in-plane stage pairs of the slab variant: 512^2 and 256^2 planes,
// complex (forward x then y; inverse y then x) and real (forward R2C x split
// then y; inverse y then C2R x merge, which also serves the Poisson solve).
#include "gbfft_plane.cuh"

namespace gbfft {

void register_plane_group_0(std::vector<PlaneKernel>& v) {
  v.push_back(make_plane_entry<512, -1, kPlain, 512, -1, kPlain>());
  v.push_back(make_plane_entry<512, 1, kPlain, 512, 1, kPlain>());
  v.push_back(make_plane_entry<256, -1, kR2CPost, 512, -1, kPlain>());
  v.push_back(make_plane_entry<512, 1, kPlain, 256, 1, kC2RPre>());
  v.push_back(make_plane_entry<256, -1, kPlain, 256, -1, kPlain>());
  v.push_back(make_plane_entry<256, 1, kPlain, 256, 1, kPlain>());
  v.push_back(make_plane_entry<128, -1, kR2CPost, 256, -1, kPlain>());
  v.push_back(make_plane_entry<256, 1, kPlain, 128, 1, kC2RPre>());
}

}  // namespace gbfft
