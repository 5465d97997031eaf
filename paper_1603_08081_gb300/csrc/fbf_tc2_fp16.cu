// Instantiations of the second tensor-core layout for the split FP16 form
// (data as hi + lo FP16 parts, weights FP16 once): D1 = D2, row chunks 4
// (W <= 16) and 5 (W <= 24).
#include "fbf_tc2_kernel.cuh"

namespace fbf {

fbf_status launch_tc2_fp16(const FilterArgs &a, cudaStream_t s) {
  if (a.W <= 16) return tc2::launch_cfg<0, 2, 4, 1>(a, s);
  if (a.W <= 24) return tc2::launch_cfg<0, 2, 5, 1>(a, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
