// fbf_filter_backward_noalloc: the gradient entry point for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: a host
// application whose framework has already reserved the device memory for its
// own allocator, or a real-time loop in which an allocation (which may block,
// synchronise, or fail under memory pressure) is not allowed.  This variant
// runs exactly the same three kernels as fbf_filter_backward, but takes its
// scratch from one fixed array in device memory that is part of this library
// (FBF_NOALLOC_SCRATCH_BYTES bytes, held on every GPU that loads the library
// until the process exits).  Requests that need more scratch than that are
// rejected with FBF_ERR_RANGE.
//
// All calls share the one array and it keeps the last call's contents.  The
// backward passes overwrite every scratch element they later read (the (a, b)
// map is written in full by the forward pass, the extended-grid gradient in
// full by the adjoint pass), so nothing needs clearing.  Calls whose work
// overlaps on the GPU (different streams, or different host threads on the
// same device without ordering) race on the array and produce wrong results.
#include <cuda_runtime.h>

#include <cstdint>

#include "fbf_internal.h"

// The shared scratch.  In host code this name is only a stand-in for the device
// symbol: its device address is looked up (with the device current) below.
static __device__ __align__(256) unsigned char g_fbf_noalloc_scratch[FBF_NOALLOC_SCRATCH_BYTES];

namespace fbf {
namespace {

// Device address of the scratch array on the current device.  Looked up on
// every call (cudaGetSymbolAddress allocates nothing and is cheap), so that an
// address is never reused after the device was reset or the module reloaded.
fbf_status scratch_address(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_fbf_noalloc_scratch) != cudaSuccess || !p) return FBF_ERR_CUDA;
  *out = p;
  return FBF_OK;
}

}  // namespace
}  // namespace fbf

using namespace fbf;

extern "C" fbf_status fbf_filter_backward_noalloc(const fbf_params *p, const float *d_in, const float *d_gout,
                                                  const float *d_out_fwd, float *d_gin, int H, int Wd,
                                                  size_t pitch, cudaStream_t stream) {
  (void)d_out_fwd;
  FilterArgs a;
  fbf_status st = pack_filter_args(p, d_in, FBF_F32, H, Wd, pitch, d_gin, pitch, &a);
  if (st != FBF_OK) return st;
  if (H == 0 || Wd == 0) return FBF_OK;
  if (!d_gout || reinterpret_cast<uintptr_t>(d_gout) % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
  if (p->form != FBF_FORM_AUTO && p->form != FBF_FORM_FP32) return FBF_ERR_UNSUPPORTED;
  if (a.W > f32_wmax()) return FBF_ERR_RANGE;
  if (backward_scratch_bytes(H, Wd, a.W, a.border) > (size_t)FBF_NOALLOC_SCRATCH_BYTES) return FBF_ERR_RANGE;
  void *scratch = nullptr;
  st = scratch_address(&scratch);
  if (st != FBF_OK) return st;
  return launch_backward(a, d_gout, pitch, d_gin, pitch, scratch, stream);
}
