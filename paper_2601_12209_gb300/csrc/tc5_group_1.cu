// Stage-kernel instantiations whose radix-16 passes run on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory), BF16 hi/lo operand
// pairs, forward and inverse: every supported length whose radix-16
// butterflies fill 128-row operand tiles (128, 256, 384, 640, 768, 1024).
#include "gbfft_kernels.cuh"

namespace gbfft {

void register_tc5_group_1(std::vector<StageKernel>& v) {
  v.push_back(make_stage_entry<128, -1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<128, 1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<256, -1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<256, 1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<384, -1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<384, 1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<640, -1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<640, 1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<768, -1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<768, 1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<1024, -1, kPlain, kPrecBF16SplitTC5>());
  v.push_back(make_stage_entry<1024, 1, kPlain, kPrecBF16SplitTC5>());
}

}  // namespace gbfft
