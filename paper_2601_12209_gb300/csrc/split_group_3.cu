// Stage-kernel instantiations with tensor-core radix-16 passes (hi/lo split
// operands), group 3: BF16 operand pairs, forward and inverse, lengths 256, 384, 640, 768, 1024.
// Every supported length with a radix-16 pass has them.
#include "gbfft_kernels.cuh"

namespace gbfft {

void register_split_group_3(std::vector<StageKernel>& v) {
  v.push_back(make_stage_entry<256, -1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<256, 1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<384, -1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<384, 1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<640, -1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<640, 1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<768, -1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<768, 1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<1024, -1, kPlain, kPrecBF16Split>());
  v.push_back(make_stage_entry<1024, 1, kPlain, kPrecBF16Split>());
}

}  // namespace gbfft
