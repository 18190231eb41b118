// Batched persistent kernel, forward direction: complex stages of every length
// the batched configuration draws (32 ... 256, factors 2, 3, 5).
#include "gbfft_many.cuh"

namespace gbfft {

void register_many_group_0(std::vector<ManyKernel>& v) {
  v.push_back(make_many_entry<kcode(32, kPlain, -1), kcode(48, kPlain, -1), kcode(60, kPlain, -1), kcode(64, kPlain, -1), kcode(80, kPlain, -1), kcode(96, kPlain, -1), kcode(120, kPlain, -1), kcode(128, kPlain, -1), kcode(160, kPlain, -1), kcode(192, kPlain, -1), kcode(256, kPlain, -1)>());
}

}  // namespace gbfft
