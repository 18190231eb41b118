// Stage-kernel instantiations with tensor-core radix-16 passes (hi/lo split
// operands), group 0: F16 operand pairs, forward and inverse, lengths 48, 80, 128, 240.
// Every supported length with a radix-16 pass has them.
#include "gbfft_kernels.cuh"

namespace gbfft {

void register_split_group_0(std::vector<StageKernel>& v) {
  v.push_back(make_stage_entry<48, -1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<48, 1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<80, -1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<80, 1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<128, -1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<128, 1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<240, -1, kPlain, kPrecF16Split>());
  v.push_back(make_stage_entry<240, 1, kPlain, kPrecF16Split>());
}

}  // namespace gbfft
