// Tensor-core form of the fused shiftable bilateral filter (Algorithm 1) for
// uint8 images, second layout: both 1-D passes of every harmonic run on the
// 5th-generation tensor cores (tcgen05.mma kind::f16, FP32 accumulation in
// tensor memory) with the CUDA cores doing only O(1) work per pixel and
// harmonic.
//
// One persistent CTA per SM (512 threads = four groups h of four warps; warp
// w reaches TMEM lanes 32 (w % 4) ... + 31) walks tiles of 32 output columns x
// (128 - 2W) output rows.  TMEM lane r is ext row r of the tile (image row
// ty0 - W + r); thread (lane r, group h) owns, for the whole tile, the pixels
// of ext row r in a few 8-column units: its demodulation unit (the 8 output
// columns 8h .. 8h + 7, ext columns Wp + 8h ..) and up to HPG halo units
// (Wp = W rounded up to a multiple of 8, so that units are 8-column aligned).
// Per pixel it keeps the exact integer phase index m = n v mod 2T in a
// register (advanced by v each harmonic) and reads (cos, sin)(pi m / T) from
// a 16-copy table built once per CTA: no per-harmonic table and no gathers of
// pixel values.  For each harmonic n:
//
//   modulate  (cos, sin, f cos, f sin)(n w f) of the thread's pixels, the f
//             channels centred (f - T/2), rounded to 16 bits (hi, and lo =
//             the residual for the split forms), written with tcgen05.st into
//             A1[channel][part] (lane = ext row, K = ext column);
//   row MMA   D1[lane r][32 c + x] = sum over the K chunks meeting the band of
//             A1[c] (TMEM) x T_i (16 x 32 Toeplitz block in shared memory);
//   re-split  thread (r, h) reads D1 of its 8 output columns and 4 channels,
//             rounds to 16 bits and stores them as row r (K = ext row) of the
//             MN-major B operand B2[K = ext row][N = 4 x + slot] -- each
//             thread writes its own row: the transpose costs no shuffles;
//   col MMA   D2[lane r][N = 4 x + slot] = sum over the 8 K chunks of
//             C (TMEM, lane = ext row r of the output, K = ext row of the
//             input, entries w[k - r + W]) x B2 chunk: M = 128, N = 128;
//   demod     thread (r, h) reads D2 of its 8 pixels (all four channels) and
//             accumulates P += d_n (cos F_r + sin F_i), Q += d_n (cos G_r +
//             sin G_i) in registers; ext row r is output row r - W, valid for
//             W <= r < 128 - W.
//
// fhat = P / Q + T/2 is written by the thread itself: no combine pass.  The
// column Toeplitz matrix lives in TMEM (written once per CTA), so the column
// MMA reads only B2 from shared memory.
//
// Schedule (separate D1, D2): per harmonic two phases separated by CTA
// barriers --
//   (A) one thread issues the column MMAs of n while every thread modulates
//       n + 1 (A1 is free: the row MMAs of n finished before the re-split of n);
//   (B) four threads issue the row MMAs of n + 1; every thread waits for the
//       column MMAs of n (its own mbarrier wait: it reads only its own lanes),
//       demodulates n, waits for the row MMAs of n + 1 and re-splits them.
// With D1 = D2 (SHARED, when A1 needs the TMEM of D2) phase B is split in two:
// demodulate n, barrier, then the row MMAs of n + 1 and their re-split.
//
// Bounded waits: every mbarrier wait gives up after a poll limit (a launch
// argument); the CTA then agrees on the failure at the next barrier, waits
// (with the full limit) for its MMAs and TMA copy in flight, records the
// failure in the library's device error word and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fbf_common.cuh"
#include "fbf_internal.h"
#include "fbf_tc_ptx.cuh"

namespace fbf {
namespace tc2 {

using namespace tc;

constexpr int kNT = 512;           // threads per CTA
constexpr int kLanes = 128;        // TMEM lanes = ext rows per tile
constexpr int kBX = 32;            // output columns per tile
constexpr int kCopies = 16;        // trig table copies (conflict-free 8-byte gathers per half warp)
constexpr int kTrigEntries = 510;  // 2T <= 510 (T <= 255)
constexpr int kTrigBytes = (kTrigEntries + 1) * kCopies * 8;  // + the zero entry in front
constexpr int kB2Part = kLanes * 128 * 2;  // one part of B2: 128 (K) x 128 (N) x 16 bit
constexpr int kB2Group = 128 * 2 * 8;      // bytes per 8-row K group of B2 (16 N groups x 128 B)
constexpr int kBoxW = 144;                 // TMA box: 144 columns (>= 8 + KX) x 128 rows of bytes
constexpr uint32_t kMaxPolls = 1u << 22;
constexpr int kErrTimeout = 2;             // device error word bit: a bounded wait gave up

// Half window rounded up to the 8-column units of the tile (ext column Wp + x
// is output column x).
__host__ __device__ constexpr int wpad(int W) { return (W + 7) & ~7; }
// ext columns of the row pass (multiple of 16): [Wp - W, Wp + 31 + W] used.
__host__ __device__ constexpr int kx_of(int W) { return (wpad(W) + kBX + W + 15) & ~15; }
// halo units per group for a maximum of KXC row chunks
__host__ __device__ constexpr int hpg_of(int kxc) { return (2 * kxc - 4 + 3) / 4; }

struct Layout {
  size_t trig, b2, br, box, bar, bytes;
};
template <int NSPLIT, int KXC>
__host__ __device__ constexpr Layout layout() {
  constexpr int kParts = NSPLIT > 1 ? 2 : 1, kWParts = NSPLIT == 3 ? 2 : 1;
  Layout L{};
  L.trig = 0;
  L.b2 = ((size_t)kTrigBytes + 1023) & ~(size_t)1023;
  L.br = L.b2 + (size_t)kParts * kB2Part;
  L.box = (L.br + (size_t)KXC * kWParts * 1024 + 1023) & ~(size_t)1023;
  L.bar = L.box + (size_t)kBoxW * kLanes;
  L.bytes = L.bar + 64;
  return L;
}

// Launch arguments besides the FilterArgs.
struct Tc2Extra {
  unsigned int *err;     // device error word
  unsigned int polls;    // poll limit of the regular waits
  int use_tma;
};

template <int BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if (BF) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}
template <int BF>
__device__ __forceinline__ float2 unpack2(uint32_t x) {
  if (BF) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x));
  return __half22float2(*reinterpret_cast<const __half2 *>(&x));
}
// (a, b) -> 16-bit pair hi and the pair of residuals lo.
template <int BF>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
  hi = pack2<BF>(a, b);
  const float2 h = unpack2<BF>(hi);
  lo = pack2<BF>(a - h.x, b - h.y);
}
template <int BF>
__device__ __forceinline__ unsigned short to16(float x) {
  if (BF) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<const unsigned short *>(&h);
  }
  const __half h = __float2half_rn(x);
  return *reinterpret_cast<const unsigned short *>(&h);
}
template <int BF>
__device__ __forceinline__ float from16(unsigned short x) {
  if (BF) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(&x));
  return __half2float(*reinterpret_cast<const __half *>(&x));
}

// BF: 0 = FP16, 1 = BF16 operands.  NSPLIT: 1 = data hi x weights hi; 2 = data
// hi/lo x weights hi; 3 = plus data hi x weights lo.  KXC: row chunks the
// instantiation is sized for (KX = 16 KXC ext columns: W <= 16 for 4, 24 for
// 5, 32 for 6, 48 for 8).  SHARED: D1 and D2 share their TMEM columns.
template <int BF, int NSPLIT, int KXC, int SHARED>
__global__ void __launch_bounds__(kNT, 1) fbf_tc2_u8_kernel(const __grid_constant__ FilterArgs a,
                                                             const __grid_constant__ CUtensorMap tmap,
                                                             const Tc2Extra x) {
  constexpr int kParts = NSPLIT > 1 ? 2 : 1;   // data parts (hi, lo)
  constexpr int kWParts = NSPLIT == 3 ? 2 : 1; // weight parts (hi, lo)
  constexpr int HPG = hpg_of(KXC);             // halo units per thread at most
  constexpr int UPT = 1 + HPG;                 // units per thread
  constexpr int kA1Stride = 8 * KXC;           // TMEM columns per (channel, part) region of A1
  constexpr uint32_t kT = 0;                   // column Toeplitz matrix (64 columns per weight part)
  constexpr uint32_t kA1 = 64 * kWParts;
  constexpr uint32_t kD1 = SHARED ? 384 : 256, kD2 = 384;
  static_assert(kA1 + 4 * kParts * kA1Stride <= kD1, "A1 fits below D1");
  static_assert(KXC >= 2 && KXC <= 8, "row chunks");
  constexpr Layout Ly = layout<NSPLIT, KXC>();
  extern __shared__ __align__(1024) unsigned char smem[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quadrant, warp group
  const int r = 32 * q + lane;            // ext row = TMEM lane of this thread
  const int W = a.W, Wp = wpad(W), KX = kx_of(W), kcr = KX / 16;
  const int H = a.H, Wd = a.Wd, BYv = kLanes - 2 * W;
  const int twoT = a.twoT;
  const float c0 = 0.5f * a.T;  // intensity centre
  const bool reflect = a.border == FBF_BORDER_REFLECT;
  const int nunits = KX / 8, demod_u = Wp / 8 + h;

  unsigned char *trig = smem + Ly.trig;         // [zero entry][entry m = 0 .. 2T-1], 16 copies of float2
  unsigned char *B2 = smem + Ly.b2;
  unsigned char *BR = smem + Ly.br;
  unsigned char *box = smem + Ly.box;
  uint64_t *mbarR = reinterpret_cast<uint64_t *>(smem + Ly.bar);
  uint64_t *mbarC = reinterpret_cast<uint64_t *>(smem + Ly.bar + 8);
  uint64_t *mbarT = reinterpret_cast<uint64_t *>(smem + Ly.bar + 16);
  uint64_t *mbarD = reinterpret_cast<uint64_t *>(smem + Ly.bar + 24);
  uint32_t *tmem_base_s = reinterpret_cast<uint32_t *>(smem + Ly.bar + 32);
  // byte offset of entry 0 of the trig table, this lane's copy folded in
  const int tb = (int)Ly.trig + kCopies * 8;

  // ---- unit assignment: the demodulation unit, then halo unit j of group h is
  // the (h + 4 j)-th of the units left and right of the four demodulation units.
  auto halo_unit = [&](int j) -> int {
    const int k = h + 4 * j, left = Wp / 8;
    if (k < left) return k;
    const int u = k - left + Wp / 8 + 4;
    return u < nunits ? u : -1;
  };

  // ---- one-time setup -------------------------------------------------------
  if (warp == 0) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(mbarR, 4);  // one commit per row-issuing warp
    mbar_init(mbarC, 1);
    mbar_init(mbarT, 1);
    mbar_init(mbarD, 4);  // drain: one commit per MMA-issuing thread
    mbar_fence_init();
  }
  // trig table: entry m (cos, sin)(pi m / T) in 16 copies; the zero entry
  // (index -1) holds the channels of pixels outside the image (TRUNCATE).
  for (int m = tid - 1; m < twoT; m += kNT) {
    float sn = 0.f, cs = 0.f;
    if (m >= 0) sincospif((float)m / a.T, &sn, &cs);
    unsigned char *ent = trig + kCopies * 8 + m * kCopies * 8;
#pragma unroll
    for (int k = 0; k < kCopies; ++k)  // rotated so that a warp's stores spread over the banks
      *reinterpret_cast<float2 *>(ent + ((k + lane) & (kCopies - 1)) * 8) = make_float2(cs, sn);
  }
  // Row Toeplitz blocks (shared memory, K-major, 1 KB each): chunk i, output x,
  // K index k = ext column 16 i + k: tap 16 i + k - Wp - x + W.
  for (int e = tid; e < kcr * kWParts * 512; e += kNT) {
    const int blk = e >> 9, el = e & 511, n = el >> 4, k = el & 15;
    const int i = blk / kWParts, bp = blk % kWParts;
    const int t = 16 * i + k - Wp - n + W;
    const float wv = (t >= 0 && t <= 2 * W) ? a.w[t] : 0.f;
    const unsigned short hi = to16<BF>(wv);
    const unsigned short v = bp == 0 ? hi : to16<BF>(wv - from16<BF>(hi));
    const int off = (n & 7) * 16 + (n >> 3) * 256 + (k & 7) * 2 + (k >> 3) * 128;
    *reinterpret_cast<unsigned short *>(BR + (size_t)blk * 1024 + off) = v;
  }
  fence_proxy_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_base_s;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  // Column Toeplitz matrix in TMEM: lane m (output ext row), K = input ext row
  // 16 i + k: w[16 i + k - m + W] inside the band; group h writes chunks 2h, 2h+1.
  {
    const int m = r;
#pragma unroll
    for (int ii = 0; ii < 2; ++ii) {
      const int i = 2 * h + ii;
      uint32_t vh[8], vl[8] = {};
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        float wv[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int t = 16 * i + 2 * kk + e - m + W;
          wv[e] = (t >= 0 && t <= 2 * W) ? a.w[t] : 0.f;
        }
        if constexpr (kWParts == 2)
          split2<BF>(wv[0], wv[1], vh[kk], vl[kk]);
        else
          vh[kk] = pack2<BF>(wv[0], wv[1]);
      }
      tmem_st_x8(tmem + lane_base + kT + (uint32_t)(8 * i), vh);
      if constexpr (kWParts == 2) tmem_st_x8(tmem + lane_base + kT + 64 + (uint32_t)(8 * i), vl);
    }
    tmem_st_wait();
  }

  // ---- TMA box of a tile: columns from floor16(tx0 - Wp), rows from ty0 - W.
  auto tile_org = [&](int t, int &ty0, int &tx0) {
    const int ty = t / a.tiles_x;
    ty0 = ty * BYv;
    tx0 = (t - ty * a.tiles_x) * kBX;
  };
  auto box_x0 = [&](int tx0) -> int { return (tx0 - Wp) >= 0 ? ((tx0 - Wp) & ~15) : -((Wp - tx0 + 15) & ~15); };
  auto issue_tma = [&](int t) {  // one thread
    int ty0, tx0;
    tile_org(t, ty0, tx0);
    mbar_arrive_expect_tx(mbarT, (uint32_t)(kBoxW * kLanes));
    tma_load_2d(box, &tmap, box_x0(tx0), ty0 - W, mbarT);
  };
  const bool use_tma = x.use_tma != 0;
  bool tma_pending = false;
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (use_tma && blockIdx.x < a.ntiles) {
    if (tid == 0) issue_tma(blockIdx.x);
    tma_pending = true;
  }

  // ---- per-thread pixel state: per unit and pixel the byte offset of its
  // current table entry (m * 128 + copy * 8, or the zero entry), its phase
  // step (v mod 2T) * 128 (two per register), and f - c0 (FP16 pairs, exact).
  int mo[UPT][8];
  uint32_t vo[UPT][4];
  uint32_t fh[UPT][4];
  const int copy8 = (lane & (kCopies - 1)) * 8;
  const int lim = twoT * kCopies * 8;  // offset of entry 2T
  auto wrap = [&](int m) -> int { return m >= lim ? m - lim : m; };

  uint32_t phR = 0, phC = 0, phT = 0;
  bool fail = false;
  const uint32_t polls = x.polls;
  auto wait_bar = [&](uint64_t *m, uint32_t &ph) {
    if (!mbar_wait_bounded(m, ph, polls)) fail = true;
    ph ^= 1;
    fence_after_sync();
  };
  auto phase_sync = [&]() -> bool {
    fence_before_sync();
    const bool ok = __syncthreads_or(fail) == 0;
    fence_after_sync();
    return ok;
  };

  // ---- modulate harmonic n: table entries of the thread's pixels -> the 16-bit
  // channels of its units in A1.  The demodulation unit's offsets are advanced by
  // the demodulation (its entry for harmonic n is read again there), the halo
  // units' here; `first`: the demodulation unit's offsets already point at n.
  auto modulate = [&](bool first) {
#pragma unroll
    for (int uu = 0; uu < UPT; ++uu) {
      const int u = uu == 0 ? demod_u : halo_unit(uu - 1);
      if (u < 0) continue;
      float2 cs[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int off = mo[uu][j];
        if (uu == 0 && !first) off = wrap(off + (int)((j & 1) ? (vo[uu][j >> 1] >> 16) : (vo[uu][j >> 1] & 0xFFFFu)));
        cs[j] = *reinterpret_cast<const float2 *>(trig + tb + off);
        if (uu > 0) mo[uu][j] = wrap(mo[uu][j] + (int)((j & 1) ? (vo[uu][j >> 1] >> 16) : (vo[uu][j >> 1] & 0xFFFFu)));
      }
      uint32_t ch[4][kParts][4];  // [channel][part][column pair]
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&fh[uu][k]));
        const float c_a = cs[2 * k].x, s_a = cs[2 * k].y, c_b = cs[2 * k + 1].x, s_b = cs[2 * k + 1].y;
        if constexpr (kParts == 2) {
          split2<BF>(c_a, c_b, ch[0][0][k], ch[0][kParts - 1][k]);
          split2<BF>(s_a, s_b, ch[1][0][k], ch[1][kParts - 1][k]);
          split2<BF>(f2.x * c_a, f2.y * c_b, ch[2][0][k], ch[2][kParts - 1][k]);
          split2<BF>(f2.x * s_a, f2.y * s_b, ch[3][0][k], ch[3][kParts - 1][k]);
        } else {
          ch[0][0][k] = pack2<BF>(c_a, c_b);
          ch[1][0][k] = pack2<BF>(s_a, s_b);
          ch[2][0][k] = pack2<BF>(f2.x * c_a, f2.y * c_b);
          ch[3][0][k] = pack2<BF>(f2.x * s_a, f2.y * s_b);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < kParts; ++p)
          tmem_st_x4(tmem + lane_base + kA1 + (uint32_t)((c * kParts + p) * kA1Stride + 4 * u), ch[c][p][0],
                     ch[c][p][1], ch[c][p][2], ch[c][p][3]);
    }
    tmem_st_wait();
  };

  // ---- row MMAs: lane 0 of warp c issues channel c into D1[32 c ..].
  auto issue_row = [&]() {
    const int c = warp;
    const uint64_t br_desc = smem_desc(smem_u32(BR), 128, 256);
    constexpr uint32_t idesc = idesc_f16(128, 32, BF, 0, 0);
#pragma unroll
    for (int i = 0; i < KXC; ++i) {
      if (i < kcr) {
#pragma unroll
        for (int pp = 0; pp < NSPLIT; ++pp) {
          const int ap = pp == 1 ? 1 : 0, bp = pp == 2 ? 1 : 0;
          mma_ts(tmem + kD1 + (uint32_t)(32 * c), tmem + kA1 + (uint32_t)((c * kParts + ap) * kA1Stride + 8 * i),
                 br_desc + (uint64_t)(((i * kWParts + bp) * 1024) >> 4), idesc, (i > 0 || pp > 0) ? 1u : 0u);
        }
      }
    }
    mma_commit(mbarR);
  };

  // ---- column MMAs: one thread, D2 (M = 128 output lanes, N = 128) over the 8 K chunks.
  auto issue_col = [&]() {
    const uint64_t b2_desc = smem_desc(smem_u32(B2), kB2Group, 128);
    constexpr uint32_t idesc = idesc_f16(128, 128, BF, 0, 1);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int pp = 0; pp < NSPLIT; ++pp) {
        const int ap = pp == 1 ? 1 : 0, bp = pp == 2 ? 1 : 0;
        mma_ts(tmem + kD2, tmem + kT + (uint32_t)(64 * bp + 8 * i),
               b2_desc + (uint64_t)((ap * kB2Part + i * 2 * kB2Group) >> 4), idesc, (i > 0 || pp > 0) ? 1u : 0u);
      }
    mma_commit(mbarC);
  };

  // ---- re-split: D1 row r, outputs x in [8h, 8h + 8), four channels -> B2 row r,
  // N = 4 x + slot with slots (cos, f cos, sin, f sin) (channels 0, 2, 1, 3).
  auto resplit = [&]() {
    uint32_t v[4][8];
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld_x8(tmem + lane_base + kD1 + (uint32_t)(32 * c + 8 * h), v[c]);
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld_wait_dep(v[c]);
    unsigned char *row = B2 + (r & 7) * 16 + (r >> 3) * kB2Group;
#pragma unroll
    for (int g = 0; g < 4; ++g) {  // N group 4 h + g: x = 8 h + 2 g, 8 h + 2 g + 1
      uint4 hi, lo = make_uint4(0u, 0u, 0u, 0u);
      const int j0 = 2 * g, j1 = 2 * g + 1;
      if constexpr (kParts == 2) {
        split2<BF>(__uint_as_float(v[0][j0]), __uint_as_float(v[2][j0]), hi.x, lo.x);
        split2<BF>(__uint_as_float(v[1][j0]), __uint_as_float(v[3][j0]), hi.y, lo.y);
        split2<BF>(__uint_as_float(v[0][j1]), __uint_as_float(v[2][j1]), hi.z, lo.z);
        split2<BF>(__uint_as_float(v[1][j1]), __uint_as_float(v[3][j1]), hi.w, lo.w);
      } else {
        hi.x = pack2<BF>(__uint_as_float(v[0][j0]), __uint_as_float(v[2][j0]));
        hi.y = pack2<BF>(__uint_as_float(v[1][j0]), __uint_as_float(v[3][j0]));
        hi.z = pack2<BF>(__uint_as_float(v[0][j1]), __uint_as_float(v[2][j1]));
        hi.w = pack2<BF>(__uint_as_float(v[1][j1]), __uint_as_float(v[3][j1]));
      }
      *reinterpret_cast<uint4 *>(row + (4 * h + g) * 128) = hi;
      if (kParts == 2) *reinterpret_cast<uint4 *>(row + kB2Part + (4 * h + g) * 128) = lo;
    }
    fence_proxy_async_smem();
  };

  // ---- demodulate harmonic n: D2 row r, N = 32 h .. 32 h + 31 = pixels x in
  // [8h, 8h + 8) x slots (G_r, F_r, G_i, F_i); the table entries of harmonic n of
  // the demodulation unit, then its offsets advance to n + 1.
  float P[8], Q[8];
  auto demod = [&](int n) {
    uint32_t v[32];
    tmem_ld_x16(tmem + lane_base + kD2 + (uint32_t)(32 * h), *reinterpret_cast<uint32_t(*)[16]>(&v[0]));
    tmem_ld_x16(tmem + lane_base + kD2 + (uint32_t)(32 * h + 16), *reinterpret_cast<uint32_t(*)[16]>(&v[16]));
    const float dn = a.d[n];
    float2 cs[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cs[j] = *reinterpret_cast<const float2 *>(trig + tb + mo[0][j]);
      mo[0][j] = wrap(mo[0][j] + (int)((j & 1) ? (vo[0][j >> 1] >> 16) : (vo[0][j >> 1] & 0xFFFFu)));
    }
    tmem_ld_wait_dep(*reinterpret_cast<uint32_t(*)[16]>(&v[0]));
    tmem_ld_wait_dep(*reinterpret_cast<uint32_t(*)[16]>(&v[16]));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float tc = dn * cs[j].x, ts = dn * cs[j].y;
      Q[j] = fmaf(tc, __uint_as_float(v[4 * j + 0]), fmaf(ts, __uint_as_float(v[4 * j + 2]), Q[j]));
      P[j] = fmaf(tc, __uint_as_float(v[4 * j + 1]), fmaf(ts, __uint_as_float(v[4 * j + 3]), P[j]));
    }
  };

  bool ok = true;
  for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
    int ty0, tx0;
    tile_org(tile, ty0, tx0);
    const int iy = ty0 - W + r;  // image row of this thread's ext row
    if (use_tma) {
      if (mbar_wait_bounded(mbarT, phT, polls)) {
        phT ^= 1;
        tma_pending = false;
      } else {
        fail = true;  // the copy is still in flight: the exit path waits for this phase
      }
      if (!phase_sync()) {
        ok = false;
        break;
      }
    }
    // ---- load the thread's pixels: REFLECT mirrors (repeatedly, for windows
    // wider than the image); TRUNCATE marks pixels outside the image, whose
    // channels are zero (the zero table entry, f = 0, no phase step).
    {
      const int bx0 = box_x0(tx0), by0 = ty0 - W;
      bool row_in = iy >= 0 && iy < H;
      const int sy = reflect ? reflect_index(iy, H) : iy;
#pragma unroll
      for (int uu = 0; uu < UPT; ++uu) {
        const int u = uu == 0 ? demod_u : halo_unit(uu - 1);
        float fv[8];
        int vm[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int ix = tx0 - Wp + 8 * (u < 0 ? 0 : u) + j;
          bool in = row_in && ix >= 0 && ix < Wd;
          int sx = ix;
          if (reflect) {
            sx = reflect_index(ix, Wd);
            in = true;
          }
          int v = 0;
          if (in && u >= 0) {
            const int by = (reflect ? sy : iy) - by0, bx = sx - bx0;
            if (use_tma && by >= 0 && by < kLanes && bx >= 0 && bx < kBoxW)
              v = box[by * kBoxW + bx];
            else
              v = __ldg(static_cast<const unsigned char *>(a.in) + (size_t)(reflect ? sy : iy) * a.in_pitch + sx);
          }
          const bool valid = in && u >= 0;
          mo[uu][j] = valid ? copy8 : copy8 - kCopies * 8;  // entry m = 0, or the zero entry
          vm[j] = valid ? (v % twoT) * (kCopies * 8) : 0;
          fv[j] = valid ? (float)v - c0 : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          vo[uu][k] = (uint32_t)vm[2 * k] | ((uint32_t)vm[2 * k + 1] << 16);
          const __half2 f2 = __floats2half2_rn(fv[2 * k], fv[2 * k + 1]);
          fh[uu][k] = *reinterpret_cast<const uint32_t *>(&f2);
        }
      }
    }
    // every thread has read the box: the next tile's copy may overwrite it
    fence_proxy_async_smem();
    if (!phase_sync()) {
      ok = false;
      break;
    }
    if (use_tma && tile + (int)gridDim.x < a.ntiles) {
      if (tid == 0) issue_tma(tile + gridDim.x);
      tma_pending = true;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) P[j] = Q[j] = 0.f;

    // ---- prologue: harmonic 0 through the row pass and the re-split
    modulate(true);
    if (!(ok = phase_sync())) break;
    if (lane == 0 && warp < 4) issue_row();
    wait_bar(mbarR, phR);
    resplit();
    if (!(ok = phase_sync())) break;

    for (int n = 0; n < a.K; ++n) {
      const bool more = n + 1 < a.K;
      if (tid == 0) issue_col();           // C(n): B2 -> D2
      if (more) modulate(false);           // A1 <- harmonic n + 1
      if (!(ok = phase_sync())) break;
      if (SHARED) {
        wait_bar(mbarC, phC);
        demod(n);
        if (!(ok = phase_sync())) break;
        if (more) {
          if (lane == 0 && warp < 4) issue_row();  // R(n+1): A1 -> D (= D2, read)
          wait_bar(mbarR, phR);
          resplit();
        }
      } else {
        if (more && lane == 0 && warp < 4) issue_row();  // R(n+1): A1 -> D1
        wait_bar(mbarC, phC);
        demod(n);
        if (more) {
          wait_bar(mbarR, phR);  // C(n) is complete too: B2 may be rewritten
          resplit();
        }
      }
      if (!(ok = phase_sync())) break;
    }
    if (!ok) break;

    // ---- fhat = P / Q + c0 for this thread's 8 pixels of output row iy
    if (r >= W && r < kLanes - W && iy < H) {
      float *orow = reinterpret_cast<float *>(reinterpret_cast<char *>(a.out) + (size_t)iy * a.out_pitch);
      const int x0 = tx0 + 8 * h;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (x0 + j < Wd) orow[x0 + j] = P[j] / Q[j] + c0;
    }
  }

  if (!ok) {
    // A bounded wait gave up: let this CTA's MMAs and TMA copy in flight land
    // (full limit) before the TMEM is released and the CTA exits.
    if (lane == 0 && warp < 4) mma_commit(mbarD);
    if (!mbar_wait_bounded(mbarD, 0, kMaxPolls)) fail = true;
    if (tma_pending) mbar_wait_bounded(mbarT, phT, kMaxPolls);
    if (tid == 0) atomicOr(x.err, (unsigned)kErrTimeout);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace tc2
}  // namespace fbf

namespace fbf {
namespace tc2 {

// Host launcher of one instantiation: tiles of 32 x (128 - 2W), one persistent
// CTA per SM (at most one per tile), the box tensor map from the per-pointer
// cache, the shared-memory attribute set once per device.
template <int BF, int NSPLIT, int KXC, int SHARED>
fbf_status launch_cfg(const FilterArgs &a0, cudaStream_t s) {
  FilterArgs a = a0;
  const int BYv = kLanes - 2 * a.W;
  if (BYv < 1 || kx_of(a.W) > 16 * KXC) return FBF_ERR_RANGE;
  a.tiles_x = (a.Wd + kBX - 1) / kBX;
  a.ntiles = a.tiles_x * ((a.H + BYv - 1) / BYv);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FBF_ERR_CUDA;
  CUtensorMap map;
  const int use_tma = cached_box_map(a.in, a.Wd, a.H, a.in_pitch, kBoxW, kLanes, &map) ? 1 : 0;
  const int sms = sm_count(dev);
  if (sms <= 0) return FBF_ERR_CUDA;
  const int grid = a.ntiles < sms ? a.ntiles : sms;
  constexpr Layout Ly = layout<NSPLIT, KXC>();
  auto kern = fbf_tc2_u8_kernel<BF, NSPLIT, KXC, SHARED>;
  static FuncAttrOnce once;
  if (!once.done(dev)) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Ly.bytes) != cudaSuccess)
      return FBF_ERR_CUDA;
    once.set(dev);
  }
  Tc2Extra x{device_error_word(), wait_polls(), use_tma};
  if (!x.err) return FBF_ERR_CUDA;
  kern<<<grid, kNT, Ly.bytes, s>>>(a, map, x);
  return cuda_status(cudaGetLastError());
}

}  // namespace tc2
}  // namespace fbf
