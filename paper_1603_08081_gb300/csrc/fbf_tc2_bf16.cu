// Instantiation of the second tensor-core layout for the BF16 form (data and
// weights both as hi + lo BF16 parts, three products per step): D1 = D2, row
// chunks 4 (W <= 16).
#include "fbf_tc2_kernel.cuh"

namespace fbf {

fbf_status launch_tc2_bf16(const FilterArgs &a, cudaStream_t s) {
  if (a.W <= 16) return tc2::launch_cfg<1, 3, 4, 1>(a, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
