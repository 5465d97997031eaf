// Instantiation of the second tensor-core layout for the split FP16 form (data
// as hi + lo FP16 parts, weights FP16 once), for the windows beyond the first
// layout's 32: the sequential schedule (one data part in TMEM at a time,
// D1 = D2), up to W = 48.  The first layout stays the faster one for the split
// forms up to W = 32 (GB300, 2048^2, K = 17, W = 9 / 30: 0.404 / 0.824 ms
// there; 0.406 ms with both parts held in TMEM here, 1.145 ms sequential).
#include "fbf_tc2_kernel.cuh"

namespace fbf {

fbf_status launch_tc2_fp16(const FilterArgs &a, cudaStream_t s) {
  if (a.W > 32 && a.W <= 48) return tc2::launch_cfg<0, 2, 8, 1, 1>(a, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
