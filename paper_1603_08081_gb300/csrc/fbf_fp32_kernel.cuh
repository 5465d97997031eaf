// Kernel template of the fused FP32 shiftable bilateral filter for uint8 images (Algorithm 1, all K
// terms in one kernel).
//
// One CTA owns an output tile of BX x BY pixels.  It stages the tile plus a W
// halo on every side as 16-bit LUT indices in shared memory, stored transposed
// (column-major) so that both 1-D passes read conflict-free, and then runs,
// for each harmonic n = 0..K-1:
//
//   modulate   channels (cos, sin, f cos, f sin)(n omega f) are gathered from a
//              per-harmonic table indexed by the pixel value (u8 input, integer
//              T: the phase n*f mod 2T is exact in integers).  The table holds 8
//              interleaved copies so a quarter-warp's 16-byte gathers never hit
//              the same bank group, whatever the pixel values;
//   row pass   1-D FIR with the 2W+1 taps along x over the BY + 2W halo rows
//              (lane = row, each thread slides along x producing 8 outputs with
//              an 8-register rotating window), results to a shared row buffer;
//              the four channels travel as two packed f32x2 pairs, so every
//              tap is two fma.rn.f32x2 per output (half the issue slots of
//              scalar FFMA at the same FMA-pipe rate);
//   col pass   1-D FIR along y (lane = column, 8 outputs per thread);
//   demod      P += d_n (cos th_i Fr + sin th_i Fi),  Q += d_n (cos th_i Gr +
//              sin th_i Gi) in registers (the real part of c_n e^{-in w f} Fbar_n
//              + c_{-n} e^{in w f} Fbar_{-n}, c_{+-n} = d_n / 2, Sec. III).
//
// After the last harmonic the tile writes fhat = P / Q once.  Out-of-image
// halo pixels hold the reflected value (REFLECT) or a sentinel whose channels
// are all zero (TRUNCATE).
#pragma once

#include <cuda_runtime.h>

#include "fbf_common.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kCopies = 8;           // interleaved LUT copies (one per lane of a quarter-warp)
constexpr int kLutEntries = 257;     // pixel values 0..255 plus the zero sentinel
constexpr int kSentinel = 256;
constexpr int kRun = 8;              // outputs per thread in each 1-D pass

struct Layout {
  int HY, NG, HYP, HX, HXA, PT, PR;
  size_t row_off, tile_off, bytes;
};

// Shared-memory layout for a BX x BY tile with half window W <= wcap (the
// padded halo-row count HYP and the pitches depend only on the tile shape and
// wcap, so they are compile-time constants inside the kernel):
//   [LUT buffer 0][LUT buffer 1]   float4[257 * 8] each (one buffer when nbuf == 1)
//   [row buffer]                   float4[(HYP + 1) * PR], PR = BX + 1 (odd)
//   [tile]                         u16[HXA * PT], column-major, PT/2 odd; each
//                                  entry is the byte offset value * 128 of the
//                                  pixel's row in a table buffer
__host__ __device__ inline Layout make_layout(int BX, int BY, int W, int nbuf, int wcap) {
  Layout L;
  L.HY = BY + 2 * W;
  L.NG = (L.HY + 31) / 32;
  L.HYP = (BY + 2 * wcap + 31) / 32 * 32;
  L.HX = BX + 2 * W;
  L.HXA = BX + 2 * wcap + kRun;
  L.PT = L.HYP + 2;
  L.PR = BX + 1;
  const size_t lut = (size_t)nbuf * kLutEntries * kCopies * sizeof(float4);
  L.row_off = lut;
  L.tile_off = L.row_off + (size_t)(L.HYP + 1) * L.PR * sizeof(float4);
  const size_t tile = (size_t)L.HXA * L.PT * sizeof(unsigned short);
  L.bytes = L.tile_off + ((tile + 127) & ~(size_t)127);
  return L;
}

#ifndef FBF_FIR_PACKED
#define FBF_FIR_PACKED 1
#endif

typedef unsigned long long u64;

// Four channels of one pixel as two f32x2 pairs: a = (cos, sin), b = (f cos, f sin).
struct Quad {
  u64 a, b;
};

__device__ __forceinline__ float lo_f(u64 x) { return __uint_as_float((unsigned)x); }
__device__ __forceinline__ float hi_f(u64 x) { return __uint_as_float((unsigned)(x >> 32)); }
__device__ __forceinline__ u64 pack_f(float lo, float hi) {
  return (u64)__float_as_uint(lo) | ((u64)__float_as_uint(hi) << 32);
}


// d = w * v + d on both halves of an f32x2 pair (one fma.rn.f32x2, or two
// scalar FMAs when FBF_FIR_PACKED == 0).
__device__ __forceinline__ void fma2(u64 &d, u64 w, u64 v) {
#if FBF_FIR_PACKED
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(w), "l"(v));
#else
  d = pack_f(fmaf(lo_f(w), lo_f(v), lo_f(d)), fmaf(hi_f(w), hi_f(v), hi_f(d)));
#endif
}

// Table of (cos, sin, v cos, v sin)(n omega v) for v = 0..255, 8 copies each;
// lane l of a quarter-warp reads copy l.  Copies are written rotated so the 8
// stores of one value land in 8 different bank groups.
__device__ __forceinline__ void build_lut(float4 *L, int n, int twoT, float T, int tid, int nt) {
  for (int v = tid; v < 256; v += nt) {
    const int m = (n * v) % twoT;  // exact phase index: n*omega*v = pi * m / T (mod 2 pi)
    float sn, cs;
    sincospif((float)m / T, &sn, &cs);
    const float fv = (float)v;
    const float4 e = make_float4(cs, sn, fv * cs, fv * sn);
#pragma unroll
    for (int j = 0; j < kCopies; ++j) L[v * kCopies + ((j + v) & (kCopies - 1))] = e;
  }
}

// One 1-D pass of kRun outputs: acc[o] = sum_k w[k] * src(o + k), where src(p)
// is produced by `load(p)`.  The kRun-register window v holds src positions
// p == j (mod kRun); after tap k the position k is dead and is replaced by
// k + kRun.  Taps run in chunks of kRun (static register names) plus a tail
// with warp-uniform guards.  The last load reads position taps - 1 + kRun,
// which callers keep inside their buffers.  w2[k] holds tap k in both halves.
template <int TAPSC, class Load>
__device__ __forceinline__ void fir_run(const u64 *w2, int taps_rt, Load load, Quad (&acc)[kRun]) {
  const int taps = TAPSC > 0 ? TAPSC : taps_rt;  // TAPSC > 0: tap count known at compile time
  Quad v[kRun];
#pragma unroll
  for (int j = 0; j < kRun; ++j) {
    v[j] = load(j);
    acc[j].a = 0ull;
    acc[j].b = 0ull;
  }
  int k = 0;
#pragma unroll(TAPSC > 0 ? 8 : 1)
  for (; k + kRun <= taps; k += kRun) {
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const u64 wk = w2[k + j];
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        fma2(acc[o].a, wk, v[(o + j) & (kRun - 1)].a);
        fma2(acc[o].b, wk, v[(o + j) & (kRun - 1)].b);
      }
      v[j] = load(k + j + kRun);
    }
  }
#pragma unroll
  for (int j = 0; j < kRun; ++j) {
    if (k + j < taps) {
      const u64 wk = w2[k + j];
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        fma2(acc[o].a, wk, v[(o + j) & (kRun - 1)].a);
        fma2(acc[o].b, wk, v[(o + j) & (kRun - 1)].b);
      }
      v[j] = load(k + j + kRun);
    }
  }
}

// Box kernel: kRun outputs of the unweighted window sum acc[o] = sum_{k < taps}
// src(o + k), the first summed directly, each next one from the previous by
// adding the entering position and subtracting the leaving one (2 f32x2 ops
// per channel pair and output instead of `taps`; the restart every kRun outputs
// bounds the rounding drift to kRun - 1 steps).  The common factor 1/taps^2 of
// the box weights cancels in fhat = P / Q and is never applied.  Reads the
// same positions as fir_run (at most taps - 1 + kRun).
template <class Load>
__device__ __forceinline__ void box_run(int taps, Load load, Quad (&acc)[kRun]) {
  const u64 one = pack_f(1.f, 1.f), minus_one = pack_f(-1.f, -1.f);
  Quad head[kRun - 1];  // src(0 .. kRun - 2): the positions that leave the window
  Quad s{0ull, 0ull};
#pragma unroll
  for (int j = 0; j < kRun - 1; ++j) {
    head[j] = load(j);
    if (j < taps) {
      fma2(s.a, one, head[j].a);
      fma2(s.b, one, head[j].b);
    }
  }
#pragma unroll 4
  for (int k = kRun - 1; k < taps; ++k) {
    const Quad v = load(k);
    fma2(s.a, one, v.a);
    fma2(s.b, one, v.b);
  }
  acc[0] = s;
#pragma unroll
  for (int o = 1; o < kRun; ++o) {
    const Quad v = load(o - 1 + taps);
    fma2(s.a, one, v.a);
    fma2(s.b, one, v.b);
    fma2(s.a, minus_one, head[o - 1].a);
    fma2(s.b, minus_one, head[o - 1].b);
    acc[o] = s;
  }
}

// Per-tile parameters of the fused FP32 filter.  w2 / d point into the kernel
// parameter block (single image) or into shared memory (batched plan).
struct K1View {
  const unsigned char *in;
  size_t in_pitch;
  float *out;
  size_t out_pitch;
  int H, Wd, W, K, twoT, border;
  float T;
  const u64 *w2;     // taps, duplicated into f32x2 pairs
  const float *d;    // cosine coefficients
};

// One output tile (origin ty0, tx0) of the fused FP32 filter: stage, then for
// every harmonic modulate / row pass / column pass / demodulate, then write
// fhat.  `smem` is the dynamic shared memory laid out by make_layout (the
// caller owns anything placed after Layout::bytes).  BOXSUM: both passes are
// unweighted running window sums (box kernel, box_run) instead of the FIR.
template <int BX, int BY, int NT, int NBUF, int WCAP, int TAPSC, int BOXSUM = 0>
__device__ __forceinline__ void k1_tile(const K1View &a, int ty0, int tx0, unsigned char *smem) {
  static_assert(BX % 32 == 0 && BY % kRun == 0 && NT % 32 == 0, "tile shape");
  static_assert(NBUF == 1 || NBUF == 2, "one or two table buffers");
  constexpr int NW = NT / 32;
  constexpr int NXR = BX / kRun;       // row-pass x runs
  constexpr int NCG = BX / 32;         // column-pass column groups
  constexpr int NYR = BY / kRun;       // column-pass y runs
  constexpr int UPW = NCG * NYR / NW;  // column-pass units per warp
  static_assert(NCG * NYR % NW == 0, "column units must divide evenly among warps");
  constexpr int kLutStride = kLutEntries * kCopies;  // float4 per table buffer

  const int W = a.W, taps = 2 * W + 1;
  const Layout Ly = make_layout(BX, BY, W, NBUF, WCAP);
  float4 *lut = reinterpret_cast<float4 *>(smem);
  ulonglong2 *rowbuf = reinterpret_cast<ulonglong2 *>(smem + Ly.row_off);
  unsigned short *tileT = reinterpret_cast<unsigned short *>(smem + Ly.tile_off);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, cp = lane & (kCopies - 1);
  const int H = a.H, Wd = a.Wd;

  // Sentinel entry of every table buffer: zero channels (TRUNCATE outside the image).
  if (tid < NBUF * kCopies) {
    lut[(tid / kCopies) * kLutStride + kSentinel * kCopies + (tid % kCopies)] =
        make_float4(0.f, 0.f, 0.f, 0.f);
  }

  // Stage the halo tile, transposed: tileT[ex * PT + ey] (byte offsets into a table buffer).
  constexpr int kCG = (BX + 2 * WCAP + kRun + 31) / 32;  // column groups of 32 staged
  stage_tile<NT, kCG>(a.in, a.in_pitch, H, Wd, a.border, ty0 - W, tx0 - W,
                 Ly.HY, Ly.HX, Ly.HYP, Ly.HXA, tileT, Ly.PT, 1, (unsigned short)(kCopies * sizeof(float4)),
                 (unsigned short)(kSentinel * kCopies * sizeof(float4)));
  build_lut(lut, 0, a.twoT, a.T, tid, NT);
  __syncthreads();

  float P[UPW][kRun], Q[UPW][kRun];
#pragma unroll
  for (int q = 0; q < UPW; ++q)
#pragma unroll
    for (int o = 0; o < kRun; ++o) P[q][o] = Q[q][o] = 0.f;

  for (int n = 0; n < a.K; ++n) {
    // This lane's copy of the current table; tile entries are byte offsets into it.
    const char *Lc = reinterpret_cast<const char *>(lut + (NBUF == 2 ? (n & 1) * kLutStride : 0) + cp);

    // Row pass over the BY + 2W halo rows (rows >= HY are padding lanes).
    for (int u = warp; u < Ly.NG * NXR; u += NW) {
      const int g = u / NXR, xr = u - g * NXR;
      const int ey = g * 32 + lane, ox0 = xr * kRun;
      const unsigned short *tp = tileT + ox0 * Ly.PT + ey;
      const int PT = Ly.PT;
      Quad acc[kRun];
      auto ld = [&](int p) {
        const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(Lc + tp[p * PT]);
        return Quad{e.x, e.y};
      };
      if (BOXSUM)
        box_run(taps, ld, acc);
      else
        fir_run<TAPSC>(a.w2, taps, ld, acc);
      ulonglong2 *rb = rowbuf + ey * Ly.PR + ox0;
#pragma unroll
      for (int o = 0; o < kRun; ++o) rb[o] = make_ulonglong2(acc[o].a, acc[o].b);
    }
    __syncthreads();

    if (NBUF == 2 && n + 1 < a.K)
      build_lut(lut + ((n + 1) & 1) * kLutStride, n + 1, a.twoT, a.T, tid, NT);

    // Column pass + demodulation into P, Q.
    const float dn = a.d[n];
#pragma unroll
    for (int q = 0; q < UPW; ++q) {
      const int u = warp + q * NW;
      const int cg = u % NCG, yr = u / NCG;
      const int ox = cg * 32 + lane, oy0 = yr * kRun;
      const ulonglong2 *cpnt = rowbuf + oy0 * Ly.PR + ox;
      const int PR = Ly.PR;
      Quad acc[kRun];
      auto ld = [&](int p) {
        const ulonglong2 e = cpnt[p * PR];
        return Quad{e.x, e.y};
      };
      if (BOXSUM)
        box_run(taps, ld, acc);
      else
        fir_run<TAPSC>(a.w2, taps, ld, acc);
      const unsigned short *cen = tileT + (ox + W) * Ly.PT + oy0 + W;
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(Lc + cen[o]);
        const float cs = lo_f(c.x), sn = hi_f(c.x);
        P[q][o] = fmaf(dn, fmaf(cs, lo_f(acc[o].b), sn * hi_f(acc[o].b)), P[q][o]);
        Q[q][o] = fmaf(dn, fmaf(cs, lo_f(acc[o].a), sn * hi_f(acc[o].a)), Q[q][o]);
      }
    }
    __syncthreads();
    if (NBUF == 1 && n + 1 < a.K) {
      build_lut(lut, n + 1, a.twoT, a.T, tid, NT);
      __syncthreads();
    }
  }

  // fhat = P / Q, written once (IEEE division, no clamp).
  float *out = a.out;
#pragma unroll
  for (int q = 0; q < UPW; ++q) {
    const int u = warp + q * NW;
    const int cg = u % NCG, yr = u / NCG;
    const int ix = tx0 + cg * 32 + lane;
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
      const int iy = ty0 + yr * kRun + o;
      if (iy < H && ix < Wd)
        *reinterpret_cast<float *>(reinterpret_cast<char *>(out) + (size_t)iy * a.out_pitch +
                                   (size_t)ix * sizeof(float)) = P[q][o] / Q[q][o];
    }
  }
}

template <int BX, int BY, int NT, int NBUF, int WCAP, int TAPSC, int BOXSUM = 0>
__global__ void __launch_bounds__(NT, 1) fbf_fp32_u8_kernel(const __grid_constant__ FilterArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tile_y = blockIdx.x / a.tiles_x, tile_x = blockIdx.x - tile_y * a.tiles_x;
  const K1View v{static_cast<const unsigned char *>(a.in), a.in_pitch, a.out, a.out_pitch, a.H, a.Wd, a.W, a.K,
                 a.twoT, a.border, a.T, a.w2, a.d};
  k1_tile<BX, BY, NT, NBUF, WCAP, TAPSC, BOXSUM>(v, tile_y * BY, tile_x * BX, smem);
}

template <int BX, int BY, int NT, int NBUF, int WCAP, int TAPSC = 0, int BOXSUM = 0>
fbf_status launch_cfg(const FilterArgs &a0, cudaStream_t s) {
  FilterArgs a = a0;
  const Layout Ly = make_layout(BX, BY, a.W, NBUF, WCAP);
  a.tiles_x = (a.Wd + BX - 1) / BX;
  const int tiles_y = (a.H + BY - 1) / BY;
  a.ntiles = a.tiles_x * tiles_y;
  auto kern = fbf_fp32_u8_kernel<BX, BY, NT, NBUF, WCAP, TAPSC, BOXSUM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Ly.bytes);
  if (e != cudaSuccess) return FBF_ERR_CUDA;
  kern<<<a.ntiles, NT, Ly.bytes, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace

// Tile shapes: 64 x 96 outputs with two table buffers for W <= 16 (<= 227 KB
// of shared memory), 32 x 192 with one buffer for 17 <= W <= 32 (<= 222 KB),
// and for 33 <= W <= 48 32 x 128 with one buffer and a run-time tap count
// (213 KB; fbf_fp32_w33_48.cu).
// Both keep the padded halo rows of the row pass at <= 1.33x the output rows
// and split the row and column units evenly over 8 warps.  The tap count is a
// template parameter (one instantiation per W), so both FIR loops unroll
// completely.
template <int Wv>
fbf_status launch_w(const FilterArgs &a, cudaStream_t s) {
  if constexpr (Wv <= 16)
    return launch_cfg<64, 96, 256, 2, 16, 2 * Wv + 1>(a, s);
  else
    return launch_cfg<32, 192, 256, 1, 32, 2 * Wv + 1>(a, s);
}

#define FBF_K1_CASE(Wv) \
  case Wv:              \
    return launch_w<Wv>(a, s);

}  // namespace fbf
