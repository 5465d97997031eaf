// Instantiations of the second tensor-core layout for the single FP16 form
// (data and weights rounded to FP16 once): separate D1 / D2 up to W = 32 (row
// chunks 4 for W <= 16, 6 for W <= 32), D1 = D2 up to W = 48 (8 chunks).
#include "fbf_tc2_kernel.cuh"

namespace fbf {

fbf_status launch_tc2_single(const FilterArgs &a, cudaStream_t s) {
  if (a.W <= 16) return tc2::launch_cfg<0, 1, 4, 0>(a, s);
  if (a.W <= 32) return tc2::launch_cfg<0, 1, 6, 0>(a, s);
  if (a.W <= 48) return tc2::launch_cfg<0, 1, 8, 1>(a, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
