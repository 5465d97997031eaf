// C-ABI entry points for the device filter: argument validation, packing of
// the per-launch constants, and dispatch to the kernel forms.
#include <cuda_runtime.h>

#include <algorithm>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "fbf_internal.h"

// Device-side error word of the library.  Kernels that wait on a barrier or a
// flag give up after a bounded number of polls and OR a code in here.
__device__ unsigned int g_fbf_device_error = 0;

namespace fbf {

fbf_status pack_filter_args(const fbf_params *p, const void *d_in, fbf_dtype dtype, int H, int Wd,
                            size_t in_pitch, float *d_out, size_t out_pitch, FilterArgs *a) {
  if (!p || !p->coeffs || !a) return FBF_ERR_INVALID_ARGUMENT;
  if (H < 0 || Wd < 0) return FBF_ERR_INVALID_ARGUMENT;
  if (dtype != FBF_U8 && dtype != FBF_F32) return FBF_ERR_INVALID_ARGUMENT;
  const bool rec = p->spatial == FBF_SPATIAL_GAUSSIAN_RECURSIVE;
  if (p->spatial != FBF_SPATIAL_GAUSSIAN && p->spatial != FBF_SPATIAL_BOX && !rec) return FBF_ERR_INVALID_ARGUMENT;
  if (p->border != FBF_BORDER_REFLECT && p->border != FBF_BORDER_TRUNCATE) return FBF_ERR_INVALID_ARGUMENT;
  if (p->spatial == FBF_SPATIAL_GAUSSIAN && !(p->sigma_s > 0.0 && std::isfinite(p->sigma_s)))
    return FBF_ERR_INVALID_ARGUMENT;
  if (p->spatial == FBF_SPATIAL_BOX && p->W <= 0) return FBF_ERR_INVALID_ARGUMENT;
  if (rec && !(p->sigma_s > 0.0 && std::isfinite(p->sigma_s))) return FBF_ERR_INVALID_ARGUMENT;
  if (rec && !(p->sigma_s >= 0.5 && p->sigma_s <= 256.0)) return FBF_ERR_RANGE;
  const int W = rec ? 0 : resolve_window(p->spatial, p->sigma_s, p->W);
  if (W < 0) return FBF_ERR_INVALID_ARGUMENT;
  if (W > FBF_WMAX) return FBF_ERR_RANGE;
  const fbf_coeffs *c = p->coeffs;
  if (c->K < 1) return FBF_ERR_INVALID_ARGUMENT;
  if (c->K > FBF_KMAX) return FBF_ERR_RANGE;
  if (!(c->T > 0.0) || !std::isfinite(c->T)) return FBF_ERR_INVALID_ARGUMENT;
  const size_t esz = dtype == FBF_U8 ? 1 : 4;
  if (H > 0 && Wd > 0) {
    if (!d_in || !d_out) return FBF_ERR_INVALID_ARGUMENT;
    if (in_pitch < (size_t)Wd * esz || out_pitch < (size_t)Wd * sizeof(float)) return FBF_ERR_INVALID_ARGUMENT;
    if (out_pitch % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
    if (dtype == FBF_F32 && in_pitch % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
    // float rows are read and written as floats: their base pointers must be 4-byte aligned
    if (reinterpret_cast<uintptr_t>(d_out) % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
    if (dtype == FBF_F32 && reinterpret_cast<uintptr_t>(d_in) % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
    if ((size_t)H * out_pitch > ((size_t)1 << 62)) return FBF_ERR_INVALID_ARGUMENT;
  }
  if (dtype == FBF_U8) {
    // u8 phases are reduced exactly in integers: T must be an integer.
    if (c->T != std::floor(c->T) || c->T > 32767.0) return FBF_ERR_UNSUPPORTED;
  }
  std::memset(a, 0, sizeof(*a));
  a->in = d_in;
  a->in_pitch = in_pitch;
  a->out = d_out;
  a->out_pitch = out_pitch;
  a->H = H;
  a->Wd = Wd;
  a->W = W;
  a->K = c->K;
  a->T = (float)c->T;
  a->twoT = dtype == FBF_U8 ? 2 * (int)c->T : 0;
  a->border = (int)p->border;
  a->box = p->spatial == FBF_SPATIAL_BOX ? 1 : 0;
  spatial_weights(rec ? FBF_SPATIAL_BOX : p->spatial, p->sigma_s, W, a->w);
  a->rec = rec ? 1 : 0;
  if (rec) recursive_coeffs(p->sigma_s, a);
  for (int j = 0; j < 2 * W + 1; ++j) {
    unsigned int b;
    std::memcpy(&b, &a->w[j], sizeof(b));
    a->w2[j] = (unsigned long long)b | ((unsigned long long)b << 32);
  }
  for (int k = 0; k < c->K; ++k) a->d[k] = (float)c->d[k];
  return FBF_OK;
}

}  // namespace fbf

using namespace fbf;

namespace fbf {

// Launch of one packed image in the requested form (validated by the caller's
// pack_filter_args; sizes non-zero).
fbf_status launch_filter(const FilterArgs &a, fbf_form form, fbf_dtype dtype, cudaStream_t stream) {
  const bool tc = is_tc_form(form);
  if (form != FBF_FORM_AUTO && form != FBF_FORM_FP32 && !tc) return FBF_ERR_INVALID_ARGUMENT;
  if (a.rec) {  // the recursive Gaussian: FP32 form, uint8 input
    if (tc || dtype != FBF_U8) return FBF_ERR_UNSUPPORTED;
    return launch_rec_u8(a, stream);
  }
  if (dtype == FBF_F32) {
    if (tc) return FBF_ERR_UNSUPPORTED;
    if (a.W > f32_wmax()) return FBF_ERR_RANGE;
    return launch_fp32_f32(a, stream);
  }
  if (form == FBF_FORM_TC_FP16) return launch_tc_u8(a, 0, stream);
  if (form == FBF_FORM_TC_BF16) return launch_tc_u8(a, 1, stream);
  if (form == FBF_FORM_TC_FP16_SINGLE) return launch_tc_u8(a, 2, stream);
  if (form == FBF_FORM_TC_BF16_SINGLE) return launch_tc_u8(a, 3, stream);
  if (form == FBF_FORM_AUTO && auto_picks_tc(a)) return launch_tc_u8(a, 0, stream);
  return launch_fp32_u8(a, stream);
}

// AUTO: the faster of the FP32 and split tensor-core FP16 forms for the window,
// from a sweep on GB300 (2048^2 u8, K = 17, ms FP32 / TC): Gaussian W = 3
// 0.363 / 0.379, W = 4 0.391 / 0.379, W = 9 0.580 / 0.412, W = 17 0.942 /
// 0.600, W = 30 1.49 / 0.82; box (FP32 as running sums) W = 3 0.344 / 0.378,
// W = 4 0.385 / 0.379, W = 16 0.645 / 0.512, W = 17 0.700 / 0.600, W = 26
// 0.911 / 0.754.  The tensor-core cost steps with the row pass's K chunks and
// with the tile rows (112 computed for W <= 16, 96 for W <= 26, 64 above); the
// FP32 cost grows with the taps (slowly for the box sums).
bool auto_picks_tc(const FilterArgs &a) { return a.W >= 4; }

}  // namespace fbf

extern "C" fbf_status fbf_filter(const fbf_params *p, const void *d_in, fbf_dtype dtype, int H, int Wd,
                                 size_t in_pitch, float *d_out, size_t out_pitch, cudaStream_t stream) {
  FilterArgs a;
  fbf_status st = pack_filter_args(p, d_in, dtype, H, Wd, in_pitch, d_out, out_pitch, &a);
  if (st != FBF_OK) return st;
  if (H == 0 || Wd == 0) return FBF_OK;
  return launch_filter(a, p->form, dtype, stream);
}

extern "C" fbf_status fbf_filter_backward(const fbf_params *p, const float *d_in, const float *d_gout,
                                          const float *d_out_fwd, float *d_gin, int H, int Wd, size_t pitch,
                                          cudaStream_t stream) {
  (void)d_out_fwd;  // the forward is recomputed: Q is needed, not only fhat
  FilterArgs a;
  fbf_status st = pack_filter_args(p, d_in, FBF_F32, H, Wd, pitch, d_gin, pitch, &a);
  if (st != FBF_OK) return st;
  if (H == 0 || Wd == 0) return FBF_OK;
  if (!d_gout || reinterpret_cast<uintptr_t>(d_gout) % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
  if (p->form != FBF_FORM_AUTO && p->form != FBF_FORM_FP32) return FBF_ERR_UNSUPPORTED;
  if (a.W > f32_wmax()) return FBF_ERR_RANGE;
  const size_t bytes = backward_scratch_bytes(H, Wd, a.W, a.border);
  void *scratch = nullptr;
  if (scratch_alloc(&scratch, bytes, stream) != FBF_OK) return FBF_ERR_CUDA;
  st = launch_backward(a, d_gout, pitch, d_gin, pitch, scratch, stream);
  if (scratch_free(scratch, stream) != FBF_OK && st == FBF_OK) st = FBF_ERR_CUDA;
  return st;
}

extern "C" fbf_status fbf_filter_stack(const fbf_params *p, const void *d_in, fbf_dtype dtype, int N, int H,
                                       int Wd, size_t in_pitch, size_t in_image_stride, float *d_out,
                                       size_t out_pitch, size_t out_image_stride, cudaStream_t stream) {
  if (N < 0) return FBF_ERR_INVALID_ARGUMENT;
  FilterArgs a;
  fbf_status st = pack_filter_args(p, d_in, dtype, H, Wd, in_pitch, d_out, out_pitch, &a);
  if (st != FBF_OK) return st;
  if (N == 0 || H == 0 || Wd == 0) return FBF_OK;
  if (N > 1 && (in_image_stride < (size_t)H * in_pitch || out_image_stride < (size_t)H * out_pitch))
    return FBF_ERR_INVALID_ARGUMENT;
  // image i starts i strides in: float images need strides that keep 4-byte alignment
  if (N > 1 && (out_image_stride % sizeof(float) != 0 || (dtype == FBF_F32 && in_image_stride % sizeof(float) != 0)))
    return FBF_ERR_INVALID_ARGUMENT;
  if (dtype == FBF_F32 && (p->form == FBF_FORM_AUTO || p->form == FBF_FORM_FP32) && !a.rec) {
    // float images: the whole stack in one launch (chunks of at most 65535 images)
    if (a.W > f32_wmax()) return FBF_ERR_RANGE;
    for (int i0 = 0; i0 < N && st == FBF_OK; i0 += 65535) {
      a.in = static_cast<const char *>(d_in) + (size_t)i0 * in_image_stride;
      a.out = reinterpret_cast<float *>(reinterpret_cast<char *>(d_out) + (size_t)i0 * out_image_stride);
      st = launch_fp32_f32_stack(a, N - i0 < 65535 ? N - i0 : 65535, in_image_stride, out_image_stride, stream);
    }
    return st;
  }
  for (int i = 0; i < N && st == FBF_OK; ++i) {
    a.in = static_cast<const char *>(d_in) + (size_t)i * in_image_stride;
    a.out = reinterpret_cast<float *>(reinterpret_cast<char *>(d_out) + (size_t)i * out_image_stride);
    st = launch_filter(a, p->form, dtype, stream);
  }
  return st;
}

extern "C" fbf_status fbf_filter_backward_stack(const fbf_params *p, const float *d_in, const float *d_gout,
                                                float *d_gin, int N, int H, int Wd, size_t pitch,
                                                size_t image_stride, cudaStream_t stream) {
  if (N < 0) return FBF_ERR_INVALID_ARGUMENT;
  FilterArgs a;
  fbf_status st = pack_filter_args(p, d_in, FBF_F32, H, Wd, pitch, d_gin, pitch, &a);
  if (st != FBF_OK) return st;
  if (N == 0 || H == 0 || Wd == 0) return FBF_OK;
  if (!d_gout) return FBF_ERR_INVALID_ARGUMENT;
  if (N > 1 && (image_stride < (size_t)H * pitch || image_stride % sizeof(float) != 0))
    return FBF_ERR_INVALID_ARGUMENT;
  if (reinterpret_cast<uintptr_t>(d_gout) % sizeof(float) != 0) return FBF_ERR_INVALID_ARGUMENT;
  if (p->form != FBF_FORM_AUTO && p->form != FBF_FORM_FP32) return FBF_ERR_UNSUPPORTED;
  if (a.W > f32_wmax()) return FBF_ERR_RANGE;
  // The stack in chunks whose scratch stays under kStackScratch bytes, each
  // chunk one launch per pass.
  constexpr size_t kStackScratch = (size_t)1 << 30;
  const size_t per = backward_scratch_stride(H, Wd, a.W, a.border);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>({(size_t)N, (size_t)65535, kStackScratch / per}));
  void *scratch = nullptr;
  if (scratch_alloc(&scratch, per * (size_t)chunk, stream) != FBF_OK) return FBF_ERR_CUDA;
  for (int i0 = 0; i0 < N && st == FBF_OK; i0 += chunk) {
    const size_t off = (size_t)i0 * image_stride;
    a.in = reinterpret_cast<const char *>(d_in) + off;
    a.out = reinterpret_cast<float *>(reinterpret_cast<char *>(d_gin) + off);
    const float *g = reinterpret_cast<const float *>(reinterpret_cast<const char *>(d_gout) + off);
    st = launch_backward_stack(a, std::min(chunk, N - i0), image_stride, g, pitch, image_stride, a.out, pitch,
                               image_stride, scratch, per, stream);
  }
  if (scratch_free(scratch, stream) != FBF_OK && st == FBF_OK) st = FBF_ERR_CUDA;
  return st;
}

extern "C" fbf_status fbf_device_error(unsigned int *code) {
  if (!code) return FBF_ERR_INVALID_ARGUMENT;
  if (cudaDeviceSynchronize() != cudaSuccess) return FBF_ERR_CUDA;
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_fbf_device_error, sizeof(v)) != cudaSuccess) return FBF_ERR_CUDA;
  if (cudaMemcpyToSymbol(g_fbf_device_error, &zero, sizeof(zero)) != cudaSuccess) return FBF_ERR_CUDA;
  unsigned int vt = 0;
  if (tc_read_clear_error(&vt) != FBF_OK) return FBF_ERR_CUDA;
  *code = v | vt;
  return *code != 0 ? FBF_ERR_TIMEOUT : FBF_OK;
}

namespace fbf {
// Device address of g_fbf_device_error on the current device (passed to the
// kernels that record their failures through a pointer).
unsigned int *device_error_word() {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_fbf_device_error) != cudaSuccess) return nullptr;
  return static_cast<unsigned int *>(p);
}
}  // namespace fbf
