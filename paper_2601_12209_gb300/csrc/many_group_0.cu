// Batched kernel, forward direction: complex stages of every length the batched
// configuration draws (32 ... 256, factors 2, 3, 5), each with the tiles per
// ticket (1, 2 or 4) whose teams still cover its 16-pencil tile.
#include "gbfft_many.cuh"

namespace gbfft {

void register_many_group_0(std::vector<ManyKernel>& v) {
  v.push_back(make_many_entry<many_code(32, -1, 1), many_code(32, -1, 2), many_code(32, -1, 4), many_code(48, -1, 1), many_code(48, -1, 2), many_code(48, -1, 4), many_code(60, -1, 1), many_code(60, -1, 2), many_code(64, -1, 1), many_code(64, -1, 2), many_code(80, -1, 1), many_code(80, -1, 2), many_code(80, -1, 4), many_code(96, -1, 1), many_code(96, -1, 2), many_code(120, -1, 1), many_code(120, -1, 2), many_code(128, -1, 1), many_code(128, -1, 2), many_code(160, -1, 1), many_code(192, -1, 1), many_code(256, -1, 1)>());
}

}  // namespace gbfft
