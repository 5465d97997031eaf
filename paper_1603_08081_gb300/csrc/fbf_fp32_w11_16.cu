// Instantiations of the fused FP32 uint8 filter for W = 11..16.
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_w11_16(const FilterArgs &a, cudaStream_t s) {
  switch (a.W) {
    FBF_K1_CASE(11)
    FBF_K1_CASE(12)
    FBF_K1_CASE(13)
    FBF_K1_CASE(14)
    FBF_K1_CASE(15)
    FBF_K1_CASE(16)
    default:
      return FBF_ERR_RANGE;
  }
}

}  // namespace fbf
