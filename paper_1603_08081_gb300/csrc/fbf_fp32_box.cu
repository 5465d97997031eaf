// Box spatial kernel in the fused FP32 filter: both 1-D passes as running
// window sums (box_run), about 2 + (2W + 1) / 8 adds per output and channel
// pair instead of 2W + 1 FMAs.  The tap count is a run-time value, so two
// instantiations (the two tile shapes) cover every W.
#include "fbf_fp32_kernel.cuh"

namespace fbf {

fbf_status launch_fp32_u8_box(const FilterArgs &a, cudaStream_t s) {
  if (a.W <= 16) return launch_cfg<64, 96, 256, 2, 16, 0, 1>(a, s);
  if (a.W <= 32) return launch_cfg<32, 192, 256, 1, 32, 0, 1>(a, s);
  return FBF_ERR_RANGE;
}

}  // namespace fbf
