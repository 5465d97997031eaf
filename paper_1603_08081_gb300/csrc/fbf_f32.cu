// FP32-input forward filter and the hand-written adjoint (gradient with respect
// to the input image) of the shiftable bilateral filter.
//
// Forward (eq. (9) via Algorithm 1) for float images: the modulated channels
// (cos, sin, f cos, f sin)(n w f) cannot come from an 8-bit table, so each
// harmonic first writes them for every halo-tile pixel (sincospi of n f / T)
// into a transposed shared-memory channel tile; the row and column passes are
// the same rotating-window FIR as the uint8 kernel.
//
// Adjoint.  With fhat = P / Q, L = sum_i g(i) fhat(i), a = g / Q, b = g fhat / Q,
// phi_N(t) = Re sum_n d_n e^{i n w t} (eq. (6)) and
//   Fbar_n = w * (f e^{i n w f}),  Gbar_n = w * e^{i n w f}        (eq. (5)),
//   Abar_n = w^T * (a e^{-i n w f}),  Bbar_n = w^T * (b e^{-i n w f}),
// the derivative of eq. (9) with respect to f(m) is
//   dL/df(m) = Re sum_n d_n [ e^{i n w f_m} ((1 + i n w f_m) Abar_n(m) - i n w Bbar_n(m))
//                            - i n w e^{-i n w f_m} (a(m) Fbar_n(m) - b(m) Gbar_n(m)) ],
// the first bracket from f(m) as a neighbour, the second from f(m) as the
// centre.  w^T is the transpose of the bordered convolution: under TRUNCATE a
// zero-padded correlation (= convolution, w is symmetric); under REFLECT the
// zero-padded correlation evaluated on the extended grid [-W, H+W) x [-W, Wd+W)
// and folded back onto the mirrored source pixels.  Because the demodulation
// factor depends only on the source pixel, the whole per-position sum can be
// formed on the extended grid first and folded once at the end.
//
// Pass 1 (this file's forward kernel with g given) writes (a, b) per pixel to
// a scratch map; pass 2 recomputes the forward channels per tile (no storage of
// the 4K channels) next to the four adjoint channels, eight real channels per
// harmonic in two FIR sweeps; pass 3 folds (REFLECT only).
#include <cuda_runtime.h>

#include "fbf_common.cuh"
#include "fbf_fp32_kernel.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kBX = 32;       // output tile columns
constexpr int kWcapF = 32;    // window limit of the FP32-input kernels
constexpr int kNTf = 256;
constexpr int kPR = kBX + 1;  // row buffer pitch (odd, in 16-byte units)

enum { kModeForward = 0, kModeAdjoint = 1 };

struct F32Args {
  const float *g;     // upstream gradient (forward with ab != null, adjoint)
  float2 *ab;         // forward: (a, b) map out (nullable); adjoint: in
  float *gext;        // adjoint: extended-grid gradient (REFLECT) or the gradient (TRUNCATE)
  size_t g_pitch;     // bytes
  int ext_off;        // adjoint: W under REFLECT (grid origin at -W), 0 under TRUNCATE
  int ext_h, ext_w;   // adjoint: grid size
  size_t gext_pitch;  // bytes
  // a stack of equal-size images (blockIdx.y = image): byte strides between
  // images of in, out, g and gext, element stride of ab (all 0 for one image)
  size_t in_istride, out_istride, g_istride, gext_istride, ab_istride;
};

// Output tiles of kBX x BY pixels for windows up to WCAP.  WCAP = 16: BY = 64
// (fewer halo rows per output) or 32 (twice the tiles, for grids too small to
// fill the GPU with 64-row tiles); the 32-row tiles also stage the adjoint's
// (a, b) halo (zero outside the image), the 64-row tiles read it from L2.
// WCAP = 32 (windows 17..32): BY = 32 with neither f nor (a, b) staged -- the
// channel tile and the row buffer take the shared memory -- both read from L2.
template <int BY, int WCAP>
struct F32Smem {
  static constexpr int kHYP = (BY + 2 * WCAP + 31) / 32 * 32;  // padded halo rows (row-pass groups of 32)
  static constexpr int kHXA = kBX + 2 * WCAP + kRun;           // halo columns incl. the FIR over-read
  static constexpr bool kStageF = WCAP <= 16;
  static constexpr bool kStageAB = BY == 32 && WCAP <= 16;
  ulonglong2 chan[kHXA * kHYP];        // transposed channel tile, 4 channels per pixel
  ulonglong2 rowbuf[(kHYP + 1) * kPR];  // row-pass output
  float fT[kStageF ? kHXA * kHYP : 1];  // halo tile of f (forward border semantics), NaN = absent
  float2 abT[kStageAB ? kHXA * kHYP : 1];  // adjoint (a, b) halo, 32-row tiles only
};

// (a, b) of the adjoint at an image position, zero outside the image.
__device__ __forceinline__ float2 ab_at(const float2 *ab, int H, int Wd, int iy, int ix) {
  return (iy >= 0 && iy < H && ix >= 0 && ix < Wd) ? __ldg(ab + (size_t)iy * Wd + ix) : make_float2(0.f, 0.f);
}

__device__ __forceinline__ float ldf(const float *base, size_t pitch, int y, int x) {
  return __ldg(reinterpret_cast<const float *>(reinterpret_cast<const char *>(base) + (size_t)y * pitch) + x);
}

// MODE forward: out = fhat (nullable), ab = (g/Q, g fhat/Q) (nullable).
// MODE adjoint: gext = per-position gradient on the grid described by F32Args.
template <int MODE, int kBY, int WCAP>
__global__ void __launch_bounds__(kNTf, 1) fbf_f32_kernel(const __grid_constant__ FilterArgs a,
                                                          const __grid_constant__ F32Args x) {
  using Smem = F32Smem<kBY, WCAP>;
  constexpr int kHYP = Smem::kHYP, kHXA = Smem::kHXA;
  constexpr bool kStageF = Smem::kStageF;
  constexpr int NW = kNTf / 32, NXR = kBX / kRun, NYR = kBY / kRun;
  constexpr int UPW = NYR / NW;  // column units per warp (1 column group of 32)
  static_assert(NYR % NW == 0 || NW % NYR == 0, "units");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>(smem_raw);

  const int W = a.W, taps = 2 * W + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int H = a.H, Wd = a.Wd;
  const int tile_y = blockIdx.x / a.tiles_x, tile_x = blockIdx.x - tile_y * a.tiles_x;
  // this block's image of the stack
  const size_t img = blockIdx.y;
  const float *fin = reinterpret_cast<const float *>(static_cast<const char *>(a.in) + img * x.in_istride);
  float *fout = a.out ? reinterpret_cast<float *>(reinterpret_cast<char *>(a.out) + img * x.out_istride) : nullptr;
  const float *gup = x.g ? reinterpret_cast<const float *>(reinterpret_cast<const char *>(x.g) + img * x.g_istride)
                         : nullptr;
  float2 *abp = x.ab ? x.ab + img * x.ab_istride : nullptr;
  float *gext = x.gext ? reinterpret_cast<float *>(reinterpret_cast<char *>(x.gext) + img * x.gext_istride) : nullptr;
  const int off = MODE == kModeAdjoint ? x.ext_off : 0;
  const int py0 = tile_y * kBY - off, px0 = tile_x * kBX - off;  // image coords of output (0, 0)
  const int HY = kBY + 2 * W, HX = kBX + 2 * W;
  const bool reflect = a.border == FBF_BORDER_REFLECT;
  const float invT = 1.0f / a.T;

  // f at halo position (ex, ey) with the forward border semantics; NaN = absent.
  auto f_at = [&](int ex, int ey) -> float {
    float fv = __int_as_float(0x7fc00000);
    if (ey < HY && ex < HX) {
      const int iy = py0 - W + ey, ix = px0 - W + ex;
      if (reflect)
        fv = ldf(fin, a.in_pitch, reflect_index(iy, H), reflect_index(ix, Wd));
      else if (iy >= 0 && iy < H && ix >= 0 && ix < Wd)
        fv = ldf(fin, a.in_pitch, iy, ix);
    }
    return fv;
  };
  auto fT_at = [&](int e) -> float {  // staged tile, or L2 (wide windows)
    if constexpr (kStageF) return S.fT[e];
    const int ex = e / kHYP;
    return f_at(ex, e - ex * kHYP);
  };

  // Stage f and, with 32-row tiles, the adjoint's (a, b) (zero outside the image).
  constexpr bool kStageAB = MODE == kModeAdjoint && Smem::kStageAB;
  if constexpr (kStageF) {
    for (int e = tid; e < kHXA * kHYP; e += kNTf) {
      const int ex = e / kHYP, ey = e - ex * kHYP;
      float2 abv = make_float2(0.f, 0.f);
      if (kStageAB && ey < HY && ex < HX) {
        const int iy = py0 - W + ey, ix = px0 - W + ex;
        if (iy >= 0 && iy < H && ix >= 0 && ix < Wd) abv = abp[(size_t)iy * Wd + ix];
      }
      S.fT[e] = f_at(ex, ey);
      if constexpr (kStageAB) S.abT[e] = abv;
    }
  }
  __syncthreads();

  float acc[UPW > 0 ? UPW : 1][kRun][2];  // forward: P, Q; adjoint: neighbour, centre terms
#pragma unroll
  for (int u = 0; u < (UPW > 0 ? UPW : 1); ++u)
#pragma unroll
    for (int o = 0; o < kRun; ++o) acc[u][o][0] = acc[u][o][1] = 0.f;

  // One FIR sweep of the four channels in S.chan: row pass to S.rowbuf, column
  // pass into `res` for this thread's column units.
  auto sweep = [&](Quad (&res)[UPW > 0 ? UPW : 1][kRun]) {
    for (int u = warp; u < (kHYP / 32) * NXR; u += NW) {
      const int g = u / NXR, xr = u - g * NXR;
      const int ey = g * 32 + lane, ox0 = xr * kRun;
      const ulonglong2 *cp = S.chan + ox0 * kHYP + ey;
      Quad accq[kRun];
      fir_run<0>(a.w2, taps,
                 [&](int p) {
                   const ulonglong2 e = cp[p * kHYP];
                   return Quad{e.x, e.y};
                 },
                 accq);
      ulonglong2 *rb = S.rowbuf + ey * kPR + ox0;
#pragma unroll
      for (int o = 0; o < kRun; ++o) rb[o] = make_ulonglong2(accq[o].a, accq[o].b);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (UPW > 0 ? UPW : 1); ++q) {
      const int yr = warp + q * NW;
      if (yr < NYR) {
        const ulonglong2 *cpn = S.rowbuf + yr * kRun * kPR + lane;
        fir_run<0>(a.w2, taps,
                   [&](int p) {
                     const ulonglong2 e = cpn[p * kPR];
                     return Quad{e.x, e.y};
                   },
                   res[q]);
      }
    }
  };

  for (int n = 0; n < a.K; ++n) {
    const float dn = a.d[n];
    const float nw = (float)n * 3.14159265358979323846f * invT;  // n * omega
    // ---- forward channels (cos, sin, f cos, f sin)(n w f) of every halo pixel.
    for (int e = tid; e < kHXA * kHYP; e += kNTf) {
      const float fv = fT_at(e);
      float sn = 0.f, cs = 0.f, fval = 0.f;
      if (fv == fv) {  // present
        sincospif((float)n * fv * invT, &sn, &cs);
        fval = fv;
      }
      S.chan[e] = make_ulonglong2(pack_f(cs, sn), pack_f(fval * cs, fval * sn));
    }
    __syncthreads();
    Quad fwd[UPW > 0 ? UPW : 1][kRun];
    sweep(fwd);
    // Centre phase (cos, sin)(n w f) of every output pixel of this thread.
#pragma unroll
    for (int q = 0; q < (UPW > 0 ? UPW : 1); ++q) {
      const int yr = warp + q * NW;
      if (yr >= NYR) continue;
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        const ulonglong2 c = S.chan[(lane + W) * kHYP + yr * kRun + o + W];
        const float cs = lo_f(c.x), sn = hi_f(c.x);
        const float Gr = lo_f(fwd[q][o].a), Gi = hi_f(fwd[q][o].a);
        const float Fr = lo_f(fwd[q][o].b), Fi = hi_f(fwd[q][o].b);
        if (MODE == kModeForward) {
          acc[q][o][0] = fmaf(dn, fmaf(cs, Fr, sn * Fi), acc[q][o][0]);  // P
          acc[q][o][1] = fmaf(dn, fmaf(cs, Gr, sn * Gi), acc[q][o][1]);  // Q
        } else {
          // centre term: d_n n w (cos V_i - sin V_r), V = a Fbar - b Gbar
          float2 abv;
          if constexpr (kStageAB)
            abv = S.abT[(lane + W) * kHYP + yr * kRun + o + W];
          else
            abv = ab_at(abp, H, Wd, py0 + yr * kRun + o, px0 + lane);
          const float Vr = abv.x * Fr - abv.y * Gr, Vi = abv.x * Fi - abv.y * Gi;
          acc[q][o][1] = fmaf(dn * nw, cs * Vi - sn * Vr, acc[q][o][1]);
        }
      }
    }
    __syncthreads();
    if (MODE == kModeAdjoint) {
      // ---- adjoint channels: (a cos, -a sin, b cos, -b sin)(n w f), zero outside
      // the image, from the forward channels in place (their cos, sin).
      for (int e = tid; e < kHXA * kHYP; e += kNTf) {
        const int ex = e / kHYP, ey = e - ex * kHYP;
        float2 abv;
        if constexpr (kStageAB)
          abv = S.abT[e];
        else
          abv = ab_at(abp, H, Wd, py0 - W + ey, px0 - W + ex);
        const u64 c = S.chan[e].x;
        const float cs = lo_f(c), sn = hi_f(c);
        S.chan[e] = make_ulonglong2(pack_f(abv.x * cs, -abv.x * sn), pack_f(abv.y * cs, -abv.y * sn));
      }
      __syncthreads();
      Quad adj[UPW > 0 ? UPW : 1][kRun];
      sweep(adj);
#pragma unroll
      for (int q = 0; q < (UPW > 0 ? UPW : 1); ++q) {
        const int yr = warp + q * NW;
        if (yr >= NYR) continue;
#pragma unroll
        for (int o = 0; o < kRun; ++o) {
          const float fm = fT_at((lane + W) * kHYP + yr * kRun + o + W);
          float sn = 0.f, cs = 0.f;
          if (fm == fm) sincospif((float)n * fm * invT, &sn, &cs);
          const float Ar = lo_f(adj[q][o].a), Ai = hi_f(adj[q][o].a);
          const float Br = lo_f(adj[q][o].b), Bi = hi_f(adj[q][o].b);
          // u = (1 + i n w f) A - i n w B;  Re[(cos + i sin) u]
          const float ur = Ar - nw * fm * Ai + nw * Bi;
          const float ui = Ai + nw * fm * Ar - nw * Br;
          acc[q][o][0] = fmaf(dn, cs * ur - sn * ui, acc[q][o][0]);
        }
      }
      __syncthreads();
    }
  }

  // ---- outputs
#pragma unroll
  for (int q = 0; q < (UPW > 0 ? UPW : 1); ++q) {
    const int yr = warp + q * NW;
    if (yr >= NYR) continue;
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
      const int oy = yr * kRun + o, ox = lane;
      if (MODE == kModeForward) {
        const int iy = py0 + oy, ix = px0 + ox;
        if (iy < H && ix < Wd) {
          const float P = acc[q][o][0], Q = acc[q][o][1];
          const float fh = P / Q;
          if (fout)
            *reinterpret_cast<float *>(reinterpret_cast<char *>(fout) + (size_t)iy * a.out_pitch +
                                       (size_t)ix * sizeof(float)) = fh;
          if (abp) {
            const float gv = ldf(gup, x.g_pitch, iy, ix);
            abp[(size_t)iy * Wd + ix] = make_float2(gv / Q, gv * fh / Q);
          }
        }
      } else {
        const int gy = tile_y * kBY + oy, gx = tile_x * kBX + ox;  // grid coordinates
        if (gy < x.ext_h && gx < x.ext_w) {
          const int iy = gy - off, ix = gx - off;
          const bool inside = iy >= 0 && iy < H && ix >= 0 && ix < Wd;
          const float v = acc[q][o][0] + (inside ? acc[q][o][1] : 0.f);
          *reinterpret_cast<float *>(reinterpret_cast<char *>(gext) + (size_t)gy * x.gext_pitch +
                                     (size_t)gx * sizeof(float)) = v;
        }
      }
    }
  }
}

// grad(m) = sum over extended positions p with reflect(p) = m of gext(p).
__global__ void fbf_fold_kernel(const float *__restrict__ gext0, size_t gext_pitch, size_t gext_istride, int W, int H,
                                int Wd, float *grad0, size_t grad_pitch, size_t grad_istride) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= Wd) return;
  const float *gext = reinterpret_cast<const float *>(reinterpret_cast<const char *>(gext0) + blockIdx.z * gext_istride);
  float *grad = reinterpret_cast<float *>(reinterpret_cast<char *>(grad0) + blockIdx.z * grad_istride);
  for (int iy = blockIdx.y; iy < H; iy += gridDim.y) {
  float s = 0.f;
  // Preimages of m in [-W, N + W): p = m + 2kN and p = -1 - m + 2kN.
  const int ky = W / (2 * H) + 1, kx = W / (2 * Wd) + 1;
  for (int sy = 0; sy < 2; ++sy)
    for (int k1 = -ky; k1 <= ky; ++k1) {
      const int py = (sy ? -1 - iy : iy) + 2 * k1 * H;
      if (py < -W || py >= H + W) continue;
      for (int sx = 0; sx < 2; ++sx)
        for (int k2 = -kx; k2 <= kx; ++k2) {
          const int px = (sx ? -1 - ix : ix) + 2 * k2 * Wd;
          if (px < -W || px >= Wd + W) continue;
          s += *(reinterpret_cast<const float *>(reinterpret_cast<const char *>(gext) + (size_t)(py + W) * gext_pitch) +
                 (px + W));
        }
    }
  *reinterpret_cast<float *>(reinterpret_cast<char *>(grad) + (size_t)iy * grad_pitch + (size_t)ix * sizeof(float)) = s;
  }
}

template <int MODE, int BY, int WCAP>
fbf_status launch_f32_by(const FilterArgs &a0, const F32Args &x, int grid_h, int grid_w, int nimg, cudaStream_t s) {
  FilterArgs a = a0;
  a.tiles_x = (grid_w + kBX - 1) / kBX;
  a.ntiles = a.tiles_x * ((grid_h + BY - 1) / BY);
  auto kern = fbf_f32_kernel<MODE, BY, WCAP>;
  const size_t smem = sizeof(F32Smem<BY, WCAP>);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FBF_ERR_CUDA;
  kern<<<dim3(a.ntiles, nimg), kNTf, smem, s>>>(a, x);
  return cuda_status(cudaGetLastError());
}

// 64-row tiles when they give at least two tiles per SM (over all images of
// the stack), else 32-row tiles (2048^2: forward 1.65 -> 1.34 ms with 64 rows;
// one 512^2 image has only 128 such tiles for 152 SMs).
template <int MODE>
fbf_status launch_f32(const FilterArgs &a, const F32Args &x, int grid_h, int grid_w, int nimg, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FBF_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nimg < 1 || nimg > 65535) return FBF_ERR_INVALID_ARGUMENT;
  if (a.W > 16) return launch_f32_by<MODE, 32, 32>(a, x, grid_h, grid_w, nimg, s);
  const long long tiles64 = (long long)((grid_w + kBX - 1) / kBX) * ((grid_h + 63) / 64) * nimg;
  if (tiles64 >= 2LL * sms) return launch_f32_by<MODE, 64, 16>(a, x, grid_h, grid_w, nimg, s);
  return launch_f32_by<MODE, 32, 16>(a, x, grid_h, grid_w, nimg, s);
}

}  // namespace

int f32_wmax() { return kWcapF; }

fbf_status launch_fp32_f32(const FilterArgs &a, cudaStream_t s) { return launch_fp32_f32_stack(a, 1, 0, 0, s); }

fbf_status launch_fp32_f32_stack(const FilterArgs &a, int n, size_t in_istride, size_t out_istride, cudaStream_t s) {
  if (a.W > kWcapF) return FBF_ERR_RANGE;
  F32Args x{};
  x.in_istride = in_istride;
  x.out_istride = out_istride;
  return launch_f32<kModeForward>(a, x, a.H, a.Wd, n, s);
}

size_t backward_scratch_bytes(int H, int Wd, int W, int border) {
  const size_t ab = (size_t)H * Wd * sizeof(float2);
  const size_t ge = border == FBF_BORDER_REFLECT ? (size_t)(H + 2 * W) * (Wd + 2 * W) * sizeof(float) : 0;
  return ((ab + 255) & ~(size_t)255) + ge;
}

size_t backward_scratch_stride(int H, int Wd, int W, int border) {
  return (backward_scratch_bytes(H, Wd, W, border) + 255) & ~(size_t)255;
}

fbf_status launch_backward(const FilterArgs &a, const float *g, size_t g_pitch, float *gin, size_t gin_pitch,
                           void *scratch, cudaStream_t s) {
  return launch_backward_stack(a, 1, 0, g, g_pitch, 0, gin, gin_pitch, 0, scratch, 0, s);
}

fbf_status launch_backward_stack(const FilterArgs &a, int n, size_t in_istride, const float *g, size_t g_pitch,
                                 size_t g_istride, float *gin, size_t gin_pitch, size_t gin_istride, void *scratch,
                                 size_t scratch_istride, cudaStream_t s) {
  if (a.rec) return FBF_ERR_UNSUPPORTED;  // the adjoint has the FIR kernels only
  if (a.W > kWcapF) return FBF_ERR_RANGE;
  if (n < 1 || n > 65535 || scratch_istride % 256 != 0) return FBF_ERR_INVALID_ARGUMENT;
  const int H = a.H, Wd = a.Wd, W = a.W;
  float2 *ab = static_cast<float2 *>(scratch);
  const size_t ab_bytes = (((size_t)H * Wd * sizeof(float2)) + 255) & ~(size_t)255;
  // Pass 1: forward with (a, b) out.
  F32Args x1{};
  x1.g = g;
  x1.g_pitch = g_pitch;
  x1.ab = ab;
  x1.in_istride = in_istride;
  x1.g_istride = g_istride;
  x1.ab_istride = scratch_istride / sizeof(float2);
  FilterArgs af = a;
  af.out = nullptr;
  fbf_status st = launch_f32<kModeForward>(af, x1, H, Wd, n, s);
  if (st != FBF_OK) return st;
  // Pass 2: adjoint on the extended grid (REFLECT) or the image (TRUNCATE).
  F32Args x2{};
  x2.ab = ab;
  x2.in_istride = in_istride;
  x2.ab_istride = scratch_istride / sizeof(float2);
  if (a.border == FBF_BORDER_REFLECT) {
    x2.ext_off = W;
    x2.ext_h = H + 2 * W;
    x2.ext_w = Wd + 2 * W;
    x2.gext = reinterpret_cast<float *>(static_cast<char *>(scratch) + ab_bytes);
    x2.gext_pitch = (size_t)x2.ext_w * sizeof(float);
    x2.gext_istride = scratch_istride;
  } else {
    x2.ext_off = 0;
    x2.ext_h = H;
    x2.ext_w = Wd;
    x2.gext = gin;
    x2.gext_pitch = gin_pitch;
    x2.gext_istride = gin_istride;
  }
  st = launch_f32<kModeAdjoint>(a, x2, x2.ext_h, x2.ext_w, n, s);
  if (st != FBF_OK || a.border != FBF_BORDER_REFLECT) return st;
  // Pass 3: fold the extended grid back onto the image.
  dim3 grid((Wd + 127) / 128, H < 65535 ? H : 65535, n);
  fbf_fold_kernel<<<grid, 128, 0, s>>>(x2.gext, x2.gext_pitch, x2.gext_istride, W, H, Wd, gin, gin_pitch,
                                       gin_istride);
  return cuda_status(cudaGetLastError());
}

}  // namespace fbf
