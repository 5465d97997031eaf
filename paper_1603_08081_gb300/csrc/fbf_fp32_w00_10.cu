// Instantiations of the fused FP32 uint8 filter for W = 0..10.
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_w00_10(const FilterArgs &a, cudaStream_t s) {
  switch (a.W) {
    FBF_K1_CASE(0)
    FBF_K1_CASE(1)
    FBF_K1_CASE(2)
    FBF_K1_CASE(3)
    FBF_K1_CASE(4)
    FBF_K1_CASE(5)
    FBF_K1_CASE(6)
    FBF_K1_CASE(7)
    FBF_K1_CASE(8)
    FBF_K1_CASE(9)
    FBF_K1_CASE(10)
    default:
      return FBF_ERR_RANGE;
  }
}

}  // namespace fbf
