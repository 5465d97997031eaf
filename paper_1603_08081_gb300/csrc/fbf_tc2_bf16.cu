// Instantiation of the second tensor-core layout for the BF16 form (data and
// weights both as hi + lo BF16 parts, three products per step), for the
// windows beyond the first layout's 32: the sequential schedule (one data part
// in TMEM at a time, D1 = D2), up to W = 48.  The first layout stays the
// faster one up to W = 32 (GB300, 2048^2, K = 17: 0.433 ms there at W = 9
// against 0.478 ms with both parts held in TMEM here).
#include "fbf_tc2_kernel.cuh"

namespace fbf {

fbf_status launch_tc2_bf16(const FilterArgs &a, cudaStream_t s) {
  if (a.W > 32 && a.W <= 48) return tc2::launch_cfg<1, 3, 8, 1, 1>(a, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
