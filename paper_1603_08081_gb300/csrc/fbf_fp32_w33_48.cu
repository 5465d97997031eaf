// Instantiations of the fused FP32 uint8 filter for W = 33..48 (run-time taps).
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_w33_48(const FilterArgs &a, cudaStream_t s) {
  if (a.W < 33 || a.W > 48) return FBF_ERR_RANGE;
  return launch_wide(a, s);
}

}  // namespace fbf
