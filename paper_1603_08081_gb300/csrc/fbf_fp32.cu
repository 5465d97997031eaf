// Dispatch of the fused FP32 uint8 filter to its per-window instantiations.
#include "fbf_internal.h"

namespace fbf {

fbf_status launch_fp32_u8_w00_10(const FilterArgs &a, cudaStream_t s);
fbf_status launch_fp32_u8_w11_16(const FilterArgs &a, cudaStream_t s);
fbf_status launch_fp32_u8_w17_22(const FilterArgs &a, cudaStream_t s);
fbf_status launch_fp32_u8_w23_27(const FilterArgs &a, cudaStream_t s);
fbf_status launch_fp32_u8_w28_32(const FilterArgs &a, cudaStream_t s);
fbf_status launch_fp32_u8_box(const FilterArgs &a, cudaStream_t s);
fbf_status launch_fp32_u8_w33_48(const FilterArgs &a, cudaStream_t s);

fbf_status launch_fp32_u8(const FilterArgs &a, cudaStream_t s) {
  // Box windows from W = 3 up as running window sums (below that the FIR with a
  // compile-time tap count is faster: W = 2 0.347 vs 0.358 ms, W = 3 0.378 vs
  // 0.358 ms on 2048^2, K = 17).
  if (a.W > 32) return launch_fp32_u8_w33_48(a, s);
  if (a.box && a.W >= 3) return launch_fp32_u8_box(a, s);
  if (a.W <= 10) return launch_fp32_u8_w00_10(a, s);
  if (a.W <= 16) return launch_fp32_u8_w11_16(a, s);
  if (a.W <= 22) return launch_fp32_u8_w17_22(a, s);
  if (a.W <= 27) return launch_fp32_u8_w23_27(a, s);
  if (a.W <= 32) return launch_fp32_u8_w28_32(a, s);
  return FBF_ERR_RANGE;
}

}  // namespace fbf
