// Instantiations of the fused FP32 uint8 filter for W = 33..48 (run-time taps).
#include "fbf_fp32_kernel.cuh"

namespace fbf {

// One instantiation with run-time taps for the FIR, one for the box sums.
fbf_status launch_fp32_u8_w33_48(const FilterArgs &a, cudaStream_t s) {
  if (a.W < 33 || a.W > 48) return FBF_ERR_RANGE;
  if (a.box) return launch_cfg<32, 128, 256, 1, 48, 0, 1>(a, s);
  return launch_cfg<32, 128, 256, 1, 48, 0, 0>(a, s);
}

}  // namespace fbf
