// Instantiations of the fused FP32 uint8 filter for W = 17..22.
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_w17_22(const FilterArgs &a, cudaStream_t s) {
  switch (a.W) {
    FBF_K1_CASE(17)
    FBF_K1_CASE(18)
    FBF_K1_CASE(19)
    FBF_K1_CASE(20)
    FBF_K1_CASE(21)
    FBF_K1_CASE(22)
    default:
      return FBF_ERR_RANGE;
  }
}

}  // namespace fbf
