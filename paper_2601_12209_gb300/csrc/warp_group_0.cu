// Warp-per-pencil stage kernels: complex lengths 512 (any layout, and specialised
// for rows -> columns and columns -> columns) and 256 (any layout, and rows ->
// columns), forward and inverse; and the
// real x stages of 512-point rows (R2C, C2R) as two-for-one length-512 complex
// transforms.
#include "gbfft_warp.cuh"

namespace gbfft {

void register_warp_group_0(std::vector<WarpKernel>& v) {
  // any layout, and specialised for the pencil pipelines' rows -> columns (the forward stages)
  v.push_back(make_warp_entry<512, -1, kPlain>());
  v.push_back(make_warp_entry<512, 1, kPlain>());
  v.push_back(make_warp_entry<512, -1, kPlain, warp_io(kRow, kCol)>());
  v.push_back(make_warp_entry<512, 1, kPlain, warp_io(kRow, kCol)>());
  v.push_back(make_warp_entry<512, -1, kPlain, warp_io(kCol, kCol)>());
  v.push_back(make_warp_entry<512, 1, kPlain, warp_io(kCol, kCol)>());
  v.push_back(make_warp_entry<256, -1, kPlain>());
  v.push_back(make_warp_entry<256, 1, kPlain>());
  v.push_back(make_warp_entry<256, -1, kPlain, warp_io(kRow, kCol)>());
  v.push_back(make_warp_entry<256, 1, kPlain, warp_io(kRow, kCol)>());
  // the real x stages of 512-point rows: two rows per length-512 complex FFT
  v.push_back(make_pair_entry<512, -1>());
  v.push_back(make_pair_entry<512, 1>());
}

}  // namespace gbfft
