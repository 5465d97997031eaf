// Instantiations of the second tensor-core layout for the single BF16 form
// (data and weights rounded to BF16 once, intensities centred): the single
// FP16 form's schedule with BF16 operands.
#include "fbf_tc2_kernel.cuh"

namespace fbf {

fbf_status launch_tc2_bf16_single(const FilterArgs &a, cudaStream_t s) {
  if (a.W <= 16) return tc2::launch_cfg<1, 1, 4, 0>(a, s);
  if (a.W <= 32) return tc2::launch_cfg<1, 1, 6, 0>(a, s);
  if (a.W <= 48) return tc2::launch_cfg<1, 1, 8, 1>(a, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
