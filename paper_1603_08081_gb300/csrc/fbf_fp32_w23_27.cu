// Instantiations of the fused FP32 uint8 filter for W = 23..27.
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_w23_27(const FilterArgs &a, cudaStream_t s) {
  switch (a.W) {
    FBF_K1_CASE(23)
    FBF_K1_CASE(24)
    FBF_K1_CASE(25)
    FBF_K1_CASE(26)
    FBF_K1_CASE(27)
    default:
      return FBF_ERR_RANGE;
  }
}

}  // namespace fbf
