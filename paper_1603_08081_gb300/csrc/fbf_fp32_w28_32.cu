// Instantiations of the fused FP32 uint8 filter for W = 28..32.
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_w28_32(const FilterArgs &a, cudaStream_t s) {
  switch (a.W) {
    FBF_K1_CASE(28)
    FBF_K1_CASE(29)
    FBF_K1_CASE(30)
    FBF_K1_CASE(31)
    FBF_K1_CASE(32)
    default:
      return FBF_ERR_RANGE;
  }
}

}  // namespace fbf
