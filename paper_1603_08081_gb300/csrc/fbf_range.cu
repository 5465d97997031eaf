// fbf_local_range: the dynamic range T of an 8-bit image over the window
// Omega = [-W, W]^2 (the definition that opens Sec. III), on the device.
//
// T = max over pixels i of max(M(i) - f(i), f(i) - m(i)), with M, m the
// largest and smallest pixel of the window around i clipped to the image.
// Clipping and mirroring see the same values (a mirrored neighbour of i is an
// image pixel at most W away from i), and so does edge replication, which is
// how the tile is loaded.  A smaller T gives a smaller omega = pi / T and fewer
// cosine terms for the same sigma_r and eps (Sec. III).
//
// One CTA per 64 x 32 block of pixels: the block plus a W halo is staged in
// shared memory as packed bytes, the window maximum and minimum are taken
// separably (rows, then columns) four pixels at a time with the byte-SIMD
// intrinsics, and the block's largest local range is merged into *d_T with
// one atomicMax.
#include <cuda_runtime.h>

#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kRX = 64, kRY = 32, kRNT = 256;

__host__ __device__ inline int range_pitch_words(int W) { return (kRX + 2 * W) / 4 + 3; }
__host__ __device__ inline size_t range_smem_bytes(int W) {
  const int EY = kRY + 2 * W;
  return (size_t)EY * range_pitch_words(W) * 4 + 2ull * EY * (kRX / 4) * 4;
}

// Four bytes starting at byte offset s (0..3) of the pair (lo, hi).
__device__ __forceinline__ uint32_t bytes_at(uint32_t lo, uint32_t hi, int s) {
  return __byte_perm(lo, hi, 0x3210 + 0x1111 * s);
}

__device__ __forceinline__ uint32_t max_byte(uint32_t v) {
  const uint32_t a = __vmaxu4(v, v >> 16);
  return max(a & 0xFFu, (a >> 8) & 0xFFu);
}

__global__ void __launch_bounds__(kRNT) fbf_local_range_kernel(const unsigned char *__restrict__ in, size_t pitch,
                                                               int H, int Wd, int W, unsigned int *d_T) {
  extern __shared__ uint32_t sm[];
  const int EY = kRY + 2 * W, PW = range_pitch_words(W);
  uint32_t *tile = sm;                       // EY rows x PW words: bytes of ext columns 0 .. 4 PW - 1
  uint32_t *rmax = tile + (size_t)EY * PW;   // EY rows x 16 words: row-window maxima of the 64 outputs
  uint32_t *rmin = rmax + (size_t)EY * (kRX / 4);
  const int x0 = blockIdx.x * kRX, y0 = blockIdx.y * kRY;

  // Stage with edge replication (clamped indices).
  for (int e = threadIdx.x; e < EY * PW; e += kRNT) {
    const int ey = e / PW, wx = e - ey * PW;
    const int iy = min(max(y0 - W + ey, 0), H - 1);
    const unsigned char *row = in + (size_t)iy * pitch;
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int ix = min(max(x0 - W + 4 * wx + b, 0), Wd - 1);
      w |= (uint32_t)__ldg(row + ix) << (8 * b);
    }
    tile[e] = w;
  }
  __syncthreads();

  // Row pass: window max / min over ext columns 4 ox .. 4 ox + 3 + 2W.
  for (int e = threadIdx.x; e < EY * (kRX / 4); e += kRNT) {
    const int ey = e / (kRX / 4), ox = e - ey * (kRX / 4);
    const uint32_t *row = tile + (size_t)ey * PW + ox;
    uint32_t mx = 0u, mn = 0xFFFFFFFFu;
    uint32_t lo = row[0], hi = row[1];
    int k = 1;
    for (int t = 0; t <= 2 * W; ++t) {
      const int s = t & 3;
      if (t > 0 && s == 0) {
        lo = hi;
        hi = row[++k];
      }
      const uint32_t v = bytes_at(lo, hi, s);
      mx = __vmaxu4(mx, v);
      mn = __vminu4(mn, v);
    }
    rmax[e] = mx;
    rmin[e] = mn;
  }
  __syncthreads();

  // Column pass and the local range of the 4 pixels of each word.
  uint32_t best = 0;
  for (int e = threadIdx.x; e < kRY * (kRX / 4); e += kRNT) {
    const int oy = e / (kRX / 4), ox = e - oy * (kRX / 4);
    uint32_t mx = 0u, mn = 0xFFFFFFFFu;
    for (int t = 0; t <= 2 * W; ++t) {
      mx = __vmaxu4(mx, rmax[(oy + t) * (kRX / 4) + ox]);
      mn = __vminu4(mn, rmin[(oy + t) * (kRX / 4) + ox]);
    }
    // centre pixels: ext row oy + W, ext columns 4 ox + W ... + 3
    const uint32_t *crow = tile + (size_t)(oy + W) * PW + ox + (W >> 2);
    const uint32_t c = bytes_at(crow[0], crow[1], W & 3);
    uint32_t r = __vmaxu4(__vsubus4(mx, c), __vsubus4(c, mn));
    // only pixels inside the image count
    const int y = y0 + oy, x = x0 + 4 * ox;
    if (y >= H) r = 0u;
    const int nin = Wd - x;  // in-image pixels of this word
    if (nin < 4) r &= nin <= 0 ? 0u : (0xFFFFFFFFu >> (8 * (4 - nin)));
    best = max(best, max_byte(r));
  }
  best = __reduce_max_sync(0xFFFFFFFFu, best);
  if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(d_T, best);
}

}  // namespace
}  // namespace fbf

using namespace fbf;

extern "C" fbf_status fbf_local_range(const void *d_in, fbf_dtype dtype, int H, int Wd, size_t pitch, int W,
                                      unsigned int *d_T, cudaStream_t stream) {
  if (!d_T || H < 0 || Wd < 0 || W < 0) return FBF_ERR_INVALID_ARGUMENT;
  if (dtype != FBF_U8) return dtype == FBF_F32 ? FBF_ERR_UNSUPPORTED : FBF_ERR_INVALID_ARGUMENT;
  if (W > FBF_WMAX) return FBF_ERR_RANGE;
  if (H > 0 && Wd > 0 && (!d_in || pitch < (size_t)Wd)) return FBF_ERR_INVALID_ARGUMENT;
  if (cudaMemsetAsync(d_T, 0, sizeof(unsigned int), stream) != cudaSuccess) return FBF_ERR_CUDA;
  if (H == 0 || Wd == 0) return FBF_OK;
  const size_t smem = range_smem_bytes(W);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fbf_local_range_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return FBF_ERR_CUDA;
  const dim3 grid((Wd + kRX - 1) / kRX, (H + kRY - 1) / kRY);
  if (grid.y > 65535u) return FBF_ERR_RANGE;
  fbf_local_range_kernel<<<grid, kRNT, smem, stream>>>(static_cast<const unsigned char *>(d_in), pitch, H, Wd, W,
                                                        d_T);
  return cuda_status(cudaGetLastError());
}
