// Internal declarations shared by the library's translation units (never
// installed, never seen by callers of fbf.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <vector_types.h>

#include "fbf.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

namespace fbf {

constexpr int TAPS_MAX = 2 * FBF_WMAX + 1;

struct FilterArgs;

// Host helpers (fbf_fit.cpp).
int resolve_window(fbf_spatial_kernel spatial, double sigma_s, int W);
// Recursive Gaussian of scale sigma_s into a->rn / rm / rp / rE (unit gain).
void recursive_coeffs(double sigma_s, FilterArgs *a);
// Recursive-Gaussian filter of one u8 image (FP32; scratch stream-ordered).
fbf_status launch_rec_u8(const FilterArgs &a, cudaStream_t s);
void spatial_weights(fbf_spatial_kernel spatial, double sigma_s, int W, float *w1);

// Everything one filter launch needs, passed by value as a __grid_constant__
// kernel parameter: the taps and coefficients live in the parameter bank, so a
// call needs no device allocation and concurrent calls cannot race on them.
struct FilterArgs {
  const void *in;
  size_t in_pitch;  // bytes
  float *out;
  size_t out_pitch;  // bytes
  int H, Wd;         // image rows, columns
  int W;             // half window; taps = 2W + 1
  int K;             // number of coefficients d_0..d_{K-1}
  int twoT;          // 2T (integer T, u8 input)
  float T;           // T as float
  int border;        // fbf_border
  int tiles_x;       // tiles per image row
  int ntiles;        // tiles in the image
  int box;           // 1: box spatial kernel (all taps equal)
  float w[TAPS_MAX];  // normalised 1-D spatial taps w1[j + W]
  float d[FBF_KMAX];  // cosine coefficients, eq. (6)
  unsigned long long w2[TAPS_MAX];  // each tap duplicated into both halves of an f32x2 pair
  // Recursive Gaussian (spatial FBF_SPATIAL_GAUSSIAN_RECURSIVE, rec = 1): two
  // second-order sections per direction, section i: causal numerator rn[i][0..1],
  // anticausal numerator rm[i][0..1] (on x[k+1], x[k+2]), denominator
  // 1 + rp[i][0] z^-1 + rp[i][1] z^-2; REFLECT extension rE samples per side.
  int rec, rE;
  float rn[2][2], rm[2][2], rp[2][2];
};

// Common host-side validation + argument packing for the single-image forms.
fbf_status pack_filter_args(const fbf_params *p, const void *d_in, fbf_dtype dtype, int H,
                            int Wd, size_t in_pitch, float *d_out, size_t out_pitch,
                            FilterArgs *a);

fbf_status launch_fp32_u8(const FilterArgs &a, cudaStream_t s);
// One packed image in `form` (AUTO resolved by auto_picks_tc); sizes non-zero.
fbf_status launch_filter(const FilterArgs &a, fbf_form form, fbf_dtype dtype, cudaStream_t stream);
bool auto_picks_tc(const FilterArgs &a);
// mode: 0 = FP16 split data, 1 = BF16 split data and weights, 2 = FP16 single,
// 3 = BF16 single (second layout only).
fbf_status launch_tc_u8(const FilterArgs &a, int mode, cudaStream_t s);
inline bool is_tc_form(fbf_form f) {
  return f == FBF_FORM_TC_FP16 || f == FBF_FORM_TC_BF16 || f == FBF_FORM_TC_FP16_SINGLE || f == FBF_FORM_TC_BF16_SINGLE;
}
// launch_tc_u8 mode of a tensor-core form.
inline int tc_mode(fbf_form f) {
  return f == FBF_FORM_TC_FP16 ? 0 : f == FBF_FORM_TC_BF16 ? 1 : f == FBF_FORM_TC_FP16_SINGLE ? 2 : 3;
}
fbf_status tc_read_clear_error(unsigned int *code);

// FP32-input forward and the adjoint (fbf_f32.cu); W <= f32_wmax().
int f32_wmax();
fbf_status launch_fp32_f32(const FilterArgs &a, cudaStream_t s);
// n equal-size images, image i at byte offset i * stride of in / out: one launch.
fbf_status launch_fp32_f32_stack(const FilterArgs &a, int n, size_t in_istride, size_t out_istride, cudaStream_t s);
size_t backward_scratch_bytes(int H, int Wd, int W, int border);
// Scratch per image of a stacked backward (backward_scratch_bytes rounded to 256).
size_t backward_scratch_stride(int H, int Wd, int W, int border);
fbf_status launch_backward(const FilterArgs &a, const float *g, size_t g_pitch, float *gin, size_t gin_pitch,
                           void *scratch, cudaStream_t s);
// The backward of n equal-size images in one launch per pass: image i's input,
// upstream gradient and gradient at byte offsets i * in_istride, i * g_istride,
// i * gin_istride, its scratch at i * scratch_istride (a multiple of 256, at
// least backward_scratch_stride).
fbf_status launch_backward_stack(const FilterArgs &a, int n, size_t in_istride, const float *g, size_t g_pitch,
                                 size_t g_istride, float *gin, size_t gin_pitch, size_t gin_istride, void *scratch,
                                 size_t scratch_istride, cudaStream_t s);

inline fbf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FBF_OK : FBF_ERR_CUDA; }

// Second tensor-core layout (fbf_tc2_*.cu): FBF_ERR_UNSUPPORTED when the
// request lies outside its instantiations (the caller then runs the first one).
fbf_status launch_tc2_u8(const FilterArgs &a, int mode, cudaStream_t s);
fbf_status launch_tc2_single(const FilterArgs &a, cudaStream_t s);
fbf_status launch_tc2_bf16_single(const FilterArgs &a, cudaStream_t s);
fbf_status launch_tc2_fp16(const FilterArgs &a, cudaStream_t s);
fbf_status launch_tc2_bf16(const FilterArgs &a, cudaStream_t s);

// Work of one persistent launch of the second tensor-core layout over a batch
// of images, each with its own window, coefficients and TMA map: a list of
// (image, tile) items (sorted by the host, most expensive first) of which CTA
// b takes items b, b + gridDim.x, ...; when a CTA moves to another image it
// rebuilds the image's row Toeplitz blocks, column Toeplitz matrix and (if T
// changed) 2T-phase table before the tile's first MMA.  (A single image takes
// its arguments and TMA map from the kernel parameters instead.)
struct Tc2Batch {
  const FilterArgs *imgs;   // per image: arguments with tiles_x / ntiles of the 32 x (128 - 2W) tiling
  const CUtensorMap *maps;  // per image: TMA map of 144 x 128 boxes (64-byte aligned)
  const int *map_ok;        // per image: 1 when its map is valid, 0 for plain loads
  const int2 *items;        // (image, tile index within the image)
  int nitems;
};

// Device tables of a batch (one allocation): per-image arguments with the
// 32 x (128 - 2W) tiling, TMA maps, and the items sorted by estimated cost
// (harmonics x row chunks per tile), most expensive first, each image's tiles
// in order.  build() skips empty images; FBF_ERR_RANGE when an image's W or T
// lies outside the layout (W <= FBF_WMAX, 2T <= 510).
struct Tc2BatchTables {
  Tc2Batch b{};
  void *mem = nullptr;
  int wmax = 0;
  fbf_status build(const FilterArgs *args, int n);
  void release();
};
// One persistent launch over a batch; mode as for launch_tc_u8.
// FBF_ERR_UNSUPPORTED outside the instantiations (the single FP16 and BF16 forms).
fbf_status launch_tc2_batch(const Tc2BatchTables &t, int mode, cudaStream_t s);

// Host helpers shared by the launchers (fbf_host.cu, fbf_api.cu).
// 2-D u8 TMA map of an image with a box of bw x bh bytes, cached per (device,
// pointer, shape, pitch, box); false when TMA's 16-byte rules are not met.
bool cached_box_map(const void *ptr, int Wd, int H, size_t pitch, int bw, int bh, CUtensorMap *out);
int sm_count(int dev);                // multiprocessor count, cached per device
unsigned int *device_error_word();    // device address of the library's error word (current device)
unsigned int wait_polls();            // poll limit of the kernels' bounded waits
// Stream-ordered scratch from the library's pool on the current device (kept
// reserved between calls); free it on the same stream.
fbf_status scratch_alloc(void **p, size_t bytes, cudaStream_t s);
fbf_status scratch_free(void *p, cudaStream_t s);
// cudaFuncSetAttribute once per kernel and device (a bit per device ordinal < 64).
struct FuncAttrOnce {
  unsigned long long mask = 0;
  bool done(int dev) const { return dev >= 0 && dev < 64 && ((__atomic_load_n(&mask, __ATOMIC_ACQUIRE) >> dev) & 1); }
  void set(int dev) {
    if (dev >= 0 && dev < 64) __atomic_fetch_or(&mask, 1ull << dev, __ATOMIC_RELEASE);
  }
};

}  // namespace fbf
