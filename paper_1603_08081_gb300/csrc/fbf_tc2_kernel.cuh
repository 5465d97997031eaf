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
// It keeps each pixel's offset into the per-harmonic channel table in a
// register, and for its demodulation unit the exact integer phase index
// m = n v mod 2T (advanced by v each harmonic).  For each harmonic n:
//
//   table     entry v = 0..255 of harmonic n: (cos, sin, f cos, f sin)(n w v)
//             (times d_n in the split forms) with the f channels centred (f - T/2), rounded to 16
//             bits (hi, and lo = the residual for the split forms), in 16 or 8
//             copies (conflict-free gathers); built from the exact phase
//             n v mod 2T and a (cos, sin) table of the 2T phases (built once
//             per CTA), two harmonics ahead, into one of two buffers;
//   modulate  one table gather per pixel, byte permutes pairing neighbouring
//             columns, tcgen05.st into A1[channel][part] (lane = ext row, K =
//             ext column);
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
//             sin G_i) with (cos, sin)(n w f) in FP32 from the 2T-phase table
//             (d_n already in D2 for the split forms); ext row r is output row
//             r - W, valid for W <= r < 128 - W.
//
// fhat = P / Q + T/2 is written by the thread itself: no combine pass.  The
// column Toeplitz matrix lives in TMEM (written once per CTA), so the column
// MMA reads only B2 from shared memory.
//
// Schedule (separate D1, D2): per harmonic two phases, one CTA barrier --
//   (A) one thread issues the column MMAs of n while every thread modulates
//       n + 1 (A1 is free: the row MMAs of n finished before the re-split of n);
//       each compute warp then arrives on an mbarrier;
//   (B) four threads issue the row MMAs of n + 1 once all sixteen warps have
//       arrived; meanwhile every thread builds the table of n + 2, waits for
//       the column MMAs of n (its own mbarrier wait: it reads only its own
//       lanes), demodulates n, waits for the row MMAs of n + 1 and re-splits
//       them; the CTA barrier then ends the harmonic (B2 rewritten).
// With D1 = D2 (SHARED, when A1 needs the TMEM of D2) A ends in a CTA barrier
// and phase B is split in two: demodulate n, barrier, then the row MMAs of
// n + 1 and their re-split.
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

constexpr int kNC = 512;           // compute threads per CTA (four groups of four warps)
constexpr int kNT = kNC + 128;     // + one warpgroup of MMA / TMA issuers
constexpr int kRegCompute = 112;   // registers per thread after setmaxnreg: compute warpgroups
constexpr int kRegIssue = 24;      //   and the issuing warpgroup: 24 for D1 = D2 (W = 33..48; 4 x 112 + 24 <= 5 x 96
constexpr int kRegIssueBatch = 32; //   per SM sub-partition), 32 otherwise and in batches (4 x 112 + 32 = 5 x 96)
constexpr int kLanes = 128;        // TMEM lanes = ext rows per tile
constexpr int kBX = 32;            // output columns per tile
constexpr int kTrigEntries = 510;  // 2T <= 510 (T <= 255)
// Copies of the 2T-phase table: 16 (conflict-free 8-byte gathers per half warp)
// for the single form, 8 for the split forms (their larger B2 and channel
// tables leave no room for 16).
__host__ __device__ constexpr int trig_copies(int nsplit) { return nsplit > 1 ? 8 : 16; }
__host__ __device__ constexpr int trig_bytes(int nsplit) { return (kTrigEntries + 1) * trig_copies(nsplit) * 8; }
constexpr int kB2Part = kLanes * 128 * 2;  // one part of B2: 128 (K) x 128 (N) x 16 bit
constexpr int kB2Group = 128 * 2 * 8;      // bytes per 8-row K group of B2 (16 N groups x 128 B)
constexpr int kBoxW = 144;                 // TMA box: 144 columns (>= 8 + KX) x 128 rows of bytes
constexpr uint32_t kDrainPolls = 1u << 16;  // polls of the exit path's waits (suspending, <= 20 us each)
constexpr uint32_t kWaitHintNs = 20000;     // suspend hint of one poll
constexpr int kErrTimeout = 2;             // device error word bit: a bounded wait gave up
constexpr int kErrTmem = 4;                // device error word bit: TMEM not allocated at column 0

// Half window rounded up to the 8-column units of the tile (ext column Wp + x
// is output column x).
__host__ __device__ constexpr int wpad(int W) { return (W + 7) & ~7; }
// ext columns of the row pass (multiple of 16): [Wp - W, Wp + 31 + W] used.
__host__ __device__ constexpr int kx_of(int W) { return (wpad(W) + kBX + W + 15) & ~15; }
// halo units per group for a maximum of KXC row chunks
__host__ __device__ constexpr int hpg_of(int kxc) { return (2 * kxc - 4 + 3) / 4; }

// Channel table of one harmonic: 257 entries (v = 0..255 and the zero entry
// 256 for pixels outside the image) of 128 bytes: 16 copies of 8 bytes
// (single form: hi words of (cos, sin) and (f cos, f sin)) or 8 copies of 16
// bytes (split forms: the hi and the lo words).
constexpr int kEntry = 128;
constexpr int kT16Bytes = 257 * kEntry;
constexpr int kZeroV = 256;

struct Layout {
  size_t trig, t16, b2, br, box, bar, bytes;
};
template <int NSPLIT, int KXC>
__host__ __device__ constexpr Layout layout() {
  constexpr int kParts = NSPLIT > 1 ? 2 : 1, kWParts = NSPLIT == 3 ? 2 : 1;
  Layout L{};
  L.trig = 0;
  L.t16 = ((size_t)trig_bytes(NSPLIT) + 1023) & ~(size_t)1023;
  L.b2 = (L.t16 + 2 * (size_t)kT16Bytes + 1023) & ~(size_t)1023;
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
typedef unsigned long long u64;
// Two floats as one f32x2 register pair (first in the low half).
__device__ __forceinline__ u64 f2(float lo, float hi) {
  u64 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ u64 u2(uint32_t lo, uint32_t hi) {
  u64 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
  return d;
}
__device__ __forceinline__ float lo32(u64 x) { return __uint_as_float((uint32_t)x); }
__device__ __forceinline__ float hi32(u64 x) { return __uint_as_float((uint32_t)(x >> 32)); }
// d += a * b on both halves (fma.rn.f32x2); mul and sub likewise.
__device__ __forceinline__ void ffma2(u64 &d, u64 a, u64 b) { asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b)); }
__device__ __forceinline__ u64 fmul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
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
// 5, 32 for 6, 48 for 8).  SHARED: D1 and D2 share their TMEM columns.  SEQ
// (split forms, with SHARED): A1 holds one data part at a time -- the row MMAs
// of a harmonic run in two rounds, hi part then lo part, with the lo part
// modulated into A1 between them -- so that wide windows fit the TMEM.
// BATCH: the work source (a1 / map1 for one image, bt for a batch).
template <int BF, int NSPLIT, int KXC, int SHARED, int SEQ, bool BATCH>
__device__ __forceinline__ void tc2_body(const FilterArgs *a1, const CUtensorMap *map1, const Tc2Batch &bt,
                                         const Tc2Extra &x) {
  constexpr int kParts = NSPLIT > 1 ? 2 : 1;   // data parts (hi, lo)
  constexpr int kA1Parts = SEQ ? 1 : kParts;   // data parts held in A1 at a time
  constexpr int kCopies = trig_copies(NSPLIT);
  constexpr bool kFold = kParts == 2;          // d_n folded into the channel table (split forms)
  static_assert(!SEQ || (kParts == 2 && SHARED), "the sequential schedule is for split forms with D1 = D2");
  constexpr int kWParts = NSPLIT == 3 ? 2 : 1; // weight parts (hi, lo)
  constexpr int HPG = hpg_of(KXC);             // halo units per thread at most
  constexpr int UPT = 1 + HPG;                 // units per thread
  constexpr int kA1Stride = 8 * KXC;           // TMEM columns per (channel, part) region of A1
  constexpr uint32_t kT = 0;                   // column Toeplitz matrix (64 columns per weight part)
  constexpr uint32_t kA1 = 64 * kWParts;
  constexpr uint32_t kD1 = SHARED ? 384 : 256, kD2 = 384;
  static_assert(kA1 + 4 * kA1Parts * kA1Stride <= kD1, "A1 fits below D1");
  static_assert(KXC >= 2 && KXC <= 8, "row chunks");
  constexpr Layout Ly = layout<NSPLIT, KXC>();
  // kNoA (separate D1 / D2, windows up to 32): no CTA barrier between the
  // modulation of n + 1 and the rest of harmonic n.  The row issuers wait on
  // mbarA (one arrival per compute warp, after its A1 stores) instead; every
  // other dependence across that point is a per-thread MMA wait or the
  // barrier that ends the harmonic.  2048^2, K = 17: -3.5% at W = 9 and 15,
  // -4% at W = 17, 24 and 30 (with four row issuers; with two it gained
  // nothing from W = 17 on).
  constexpr bool kNoA = !SHARED;
  extern __shared__ __align__(1024) unsigned char smem[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // warps 0..15 compute (TMEM lane quadrant q, column group h); warps 16..19
  // only issue (lane 0): the row MMAs of channel warp - 16 each, and besides
  // warp 16 the column MMAs, warp 19 the TMA copies.  One thread issues an MMA
  // about every 50 cycles, so the small row MMAs take four issuers (-4 to -5%
  // against two), and no compute warp is held up while an issuer waits for
  // room in the MMA queue.
  const bool compute = warp < kNC / 32;
  const int q = warp & 3, h = compute ? warp >> 2 : 0;
  const int iw = warp - kNC / 32;  // issuer warp index 0..3 (compute warps: negative)
  const bool col_issuer = lane == 0 && iw == 0, row_issuer = lane == 0 && iw >= 0,
             tma_issuer = lane == 0 && iw == 3;
  const int r = 32 * q + lane;            // ext row = TMEM lane of this thread
  const int nitems = BATCH ? bt.nitems : a1->ntiles;

  unsigned char *trig = smem + Ly.trig;         // [zero entry][entry m = 0 .. 2T-1], 16 copies of float2
  unsigned char *B2 = smem + Ly.b2;
  unsigned char *BR = smem + Ly.br;
  unsigned char *box = smem + Ly.box;
  uint64_t *mbarR = reinterpret_cast<uint64_t *>(smem + Ly.bar);
  uint64_t *mbarC = reinterpret_cast<uint64_t *>(smem + Ly.bar + 8);
  uint64_t *mbarT = reinterpret_cast<uint64_t *>(smem + Ly.bar + 16);
  uint64_t *mbarD = reinterpret_cast<uint64_t *>(smem + Ly.bar + 24);
  uint32_t *tmem_base_s = reinterpret_cast<uint32_t *>(smem + Ly.bar + 32);
  uint64_t *mbarA = reinterpret_cast<uint64_t *>(smem + Ly.bar + 40);
  // byte offset of entry 0 of the trig table, this lane's copy folded in
  const int tb = (int)Ly.trig + kCopies * 8;
  const int bv = tid & 255, bhalf = tid >> 8;  // channel-table entry built by this thread

  // ---- the image of the current tile and what follows from it (one image:
  // set once; batch: when a CTA's item moves to another image)
  const FilterArgs *A = a1;
  int W = 0, Wp = 0, KX = 0, kcr = 0, H = 0, Wd = 0, BYv = 0, twoT = 2, nunits = 0, demod_u = 0, lim = 0,
      bstep = 0;
  float c0 = 0.f;  // intensity centre T / 2
  bool reflect = false;
  auto set_image = [&](const FilterArgs *p) {
    A = p;
    W = p->W;
    Wp = wpad(W);
    KX = kx_of(W);
    kcr = KX / 16;
    H = p->H;
    Wd = p->Wd;
    BYv = kLanes - 2 * W;
    twoT = p->twoT;
    c0 = 0.5f * p->T;
    reflect = p->border == FBF_BORDER_REFLECT;
    nunits = KX / 8;
    demod_u = Wp / 8 + h;
    lim = twoT * kCopies * 8;  // offset of entry 2T
    bstep = (bv % twoT) * (kCopies * 8);
  };
  set_image(BATCH ? bt.imgs + (nitems > 0 && (int)blockIdx.x < nitems ? bt.items[blockIdx.x].x : 0) : a1);

  // ---- unit assignment: the demodulation unit, then halo unit j of group h is
  // the (h + 4 j)-th of the units left and right of the four demodulation units.
  auto halo_unit = [&](int j) -> int {
    const int k = h + 4 * j, left = Wp / 8;
    if (k < left) return k;
    const int u = k - left + Wp / 8 + 4;
    return u < nunits ? u : -1;
  };

  // ---- per-image tables (threads t0, t0 + stride, ...).  trig: entry m (cos,
  // sin)(pi m / T) in 16 copies; the zero entry (index -1) holds the channels of
  // pixels outside the image (TRUNCATE).
  auto setup_trig = [&](int t0, int stride) {
    for (int m = t0 - 1; m < twoT; m += stride) {
      float sn = 0.f, cs = 0.f;
      if (m >= 0) sincospif((float)m / A->T, &sn, &cs);
      unsigned char *ent = trig + kCopies * 8 + m * kCopies * 8;
#pragma unroll
      for (int k = 0; k < kCopies; ++k)  // rotated so that a warp's stores spread over the banks
        *reinterpret_cast<float2 *>(ent + ((k + lane) & (kCopies - 1)) * 8) = make_float2(cs, sn);
    }
  };
  // Row Toeplitz blocks (shared memory, K-major, 1 KB each): chunk i, output x,
  // K index k = ext column 16 i + k: tap 16 i + k - Wp - x + W.
  // A thread's taps are loaded before any is stored (at most KXC x weight parts
  // each: stride >= 512), so that their latencies overlap when a batch's CTA
  // moves to another image.
  auto setup_row_toeplitz = [&](int t0, int stride) {
    constexpr int kMaxE = KXC * kWParts;
    const int total = kcr * kWParts * 512;
    float wv[kMaxE];
#pragma unroll
    for (int j = 0; j < kMaxE; ++j) {
      const int e = t0 + j * stride, blk = e >> 9, el = e & 511, n = el >> 4, k = el & 15;
      const int t = 16 * (blk / kWParts) + k - Wp - n + W;
      wv[j] = (e < total && t >= 0 && t <= 2 * W) ? A->w[t] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < kMaxE; ++j) {
      const int e = t0 + j * stride;
      if (e >= total) break;
      const int blk = e >> 9, el = e & 511, n = el >> 4, k = el & 15, bp = blk % kWParts;
      const unsigned short hi = to16<BF>(wv[j]);
      const unsigned short v = bp == 0 ? hi : to16<BF>(wv[j] - from16<BF>(hi));
      const int off = (n & 7) * 16 + (n >> 3) * 256 + (k & 7) * 2 + (k >> 3) * 128;
      *reinterpret_cast<unsigned short *>(BR + (size_t)blk * 1024 + off) = v;
    }
  };
  // Column Toeplitz matrix in TMEM (compute threads): lane m (output ext row),
  // K = input ext row 16 i + k: w[16 i + k - m + W] inside the band; group h
  // writes chunks 2h, 2h+1.
  constexpr uint32_t tmem = 0;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  auto setup_col_toeplitz = [&]() {
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
          wv[e] = (t >= 0 && t <= 2 * W) ? A->w[t] : 0.f;
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
  };

  // ---- one-time setup -------------------------------------------------------
  if (warp == 0) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(mbarR, 4);  // one commit per row-MMA issuer (one per issuing warp)
    mbar_init(mbarC, 1);
    mbar_init(mbarT, 1);
    mbar_init(mbarD, 4);  // drain: one commit per MMA-issuing thread
    mbar_init(mbarA, kNC / 32);  // kNoA: A1 of the next harmonic stored, one arrival per compute warp
    mbar_fence_init();
  }
  if (!BATCH) {  // one image: its tables once, by every thread (batch: per image, below)
    setup_trig(tid, kNT);
    setup_row_toeplitz(tid, kNT);
  }
  // zero entries (v = 256) of both channel-table buffers: pixels outside the image
  if (tid < 2 * kEntry / 16)
    *reinterpret_cast<uint4 *>(smem + Ly.t16 + (size_t)(tid / (kEntry / 16)) * kT16Bytes + kZeroV * kEntry +
                               (tid % (kEntry / 16)) * 16) = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  // All 512 columns are allocated, so the allocation starts at lane 0, column 0:
  // the MMA operands below are compile-time TMEM addresses (issued from uniform
  // registers).  Anything else is refused as a failed launch.
  const bool tmem_ok = *tmem_base_s == 0;
  if (!BATCH && tmem_ok && compute) setup_col_toeplitz();

  // ---- items: image and tile; the TMA box of a tile starts at column
  // floor16(tx0 - Wp) and row ty0 - W.
  auto item_image = [&](int it) -> int { return BATCH ? bt.items[it].x : 0; };
  auto item_tile = [&](int it) -> int { return BATCH ? bt.items[it].y : it; };
  auto item_tma = [&](int it) -> bool { return BATCH ? bt.map_ok[bt.items[it].x] != 0 : x.use_tma != 0; };
  auto box_x0 = [](int tx0, int wp) -> int { return (tx0 - wp) >= 0 ? ((tx0 - wp) & ~15) : -((wp - tx0 + 15) & ~15); };
  auto issue_tma = [&](int it) {  // one thread: the box of item it (any image)
    const int img = item_image(it), t = item_tile(it);
    const FilterArgs *p = BATCH ? bt.imgs + img : a1;
    const int w = p->W, by = kLanes - 2 * w, ty = t / p->tiles_x;
    const int tx0 = (t - ty * p->tiles_x) * kBX;
    mbar_arrive_expect_tx(mbarT, (uint32_t)(kBoxW * kLanes));
    tma_load_2d(box, BATCH ? static_cast<const void *>(bt.maps + img) : static_cast<const void *>(map1),
                box_x0(tx0, wpad(w)), ty * by - w, mbarT);
  };
  bool tma_pending = false;
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if ((int)blockIdx.x < nitems && item_tma(blockIdx.x)) {
    if (tma_issuer) issue_tma(blockIdx.x);
    tma_pending = true;
  }

  // ---- per-thread state.  po: per unit and pixel the byte offset of its entry
  // in a channel table (v * 128 + this lane's copy, or the zero entry).  For the
  // demodulation unit, mo: the byte offset of (cos, sin)(pi m / T) in the
  // 2T-phase table (m * 128 + copy, or its zero entry) for the current
  // harmonic, and vo: its step (v mod 2T) * 128, two per register.
  constexpr int kCp = kParts == 2 ? 8 : 16;             // table copies
  const int copy_off = kParts == 2 ? (lane & 7) * 16 : (lane & 15) * 8;
  int po[UPT][8];
  int mo[8];
  uint32_t vo[4];
  const int copy8 = (lane & (kCopies - 1)) * 8;
  auto wrap = [&](int m) -> int { return m >= lim ? m - lim : m; };
  // v mod 2T for a pixel value 0 <= v <= 255 without an integer division (inv2T
  // = 1 / 2T): the float quotient is exact to within one, and one correction
  // each way fixes it
  auto mod2T = [&](int v, float inv2T) -> int {
    int m = v - twoT * __float2int_rz((float)v * inv2T);
    if (m < 0) m += twoT;
    if (m >= twoT) m -= twoT;
    return m;
  };
  unsigned char *t16 = smem + Ly.t16;

  uint32_t phR = 0, phC = 0, phT = 0, phA = 0;
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

  // ---- channel table of harmonic n into buffer b: thread t builds entry
  // v = t % 256 (half of its copies); bm is the byte offset of its phase
  // n v mod 2T in the 2T-phase table (advanced here, harmonics in order).
  int bm = 0;
  auto build_table = [&](int n, int b) {
    const float2 cs = *reinterpret_cast<const float2 *>(trig + tb + bm + copy8);
    bm = wrap(bm + bstep);
    // the split forms fold d_n into the table; the single form keeps the plain
    // channels (rounding d_n-scaled values to FP16 once doubles its error: an
    // FP64 emulation of both on the 2048^2 image, sigma_s = 3, sigma_r = 40
    // gives 0.043 against 0.020 gray) and multiplies by d_n when demodulating
    const float dn = kFold ? A->d[n] : 1.f, fv = (float)bv - c0;
    const float dc = dn * cs.x, ds = dn * cs.y, dfc = dn * (fv * cs.x), dfs = dn * (fv * cs.y);
    unsigned char *ent = t16 + (size_t)b * kT16Bytes + bv * kEntry;
    if constexpr (kParts == 2) {
      uint4 e;
      split2<BF>(dc, ds, e.x, e.z);
      split2<BF>(dfc, dfs, e.y, e.w);
      // the two threads of an entry write disjoint halves of its copies, each
      // lane starting at its own copy (neighbouring lanes hit different banks)
#pragma unroll
      for (int k = 0; k < kCp / 2; ++k)
        *reinterpret_cast<uint4 *>(ent + ((lane + bhalf * (kCp / 2) + k) & (kCp - 1)) * 16) = e;
    } else {
      // 16-byte stores of two copies each
      const uint32_t e0 = pack2<BF>(dc, ds), e1 = pack2<BF>(dfc, dfs);
      const uint4 e = make_uint4(e0, e1, e0, e1);
#pragma unroll
      for (int k = 0; k < kCp / 4; ++k)
        *reinterpret_cast<uint4 *>(ent + ((lane + bhalf * (kCp / 4) + k) & (kCp / 2 - 1)) * 16) = e;
    }
  };

  // ---- modulate with the table in buffer b: per unit, one gather per pixel,
  // neighbouring columns paired by byte permutes, four-column TMEM stores.  SEQ:
  // only data part `part` (0 = hi, 1 = lo), into the one set of A1 regions.
  auto modulate = [&](int b, int part) {
    const unsigned char *tb16 = t16 + (size_t)b * kT16Bytes;
#pragma unroll
    for (int uu = 0; uu < UPT; ++uu) {
      const int u = uu == 0 ? demod_u : halo_unit(uu - 1);
      if (u < 0) continue;
      uint32_t ch[4][kA1Parts][4];  // [channel][part held][column pair]
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (kParts == 2) {
          const uint4 e0 = *reinterpret_cast<const uint4 *>(tb16 + po[uu][2 * k]);
          const uint4 e1 = *reinterpret_cast<const uint4 *>(tb16 + po[uu][2 * k + 1]);
          if constexpr (SEQ) {
            const uint32_t a0 = part ? e0.z : e0.x, a1 = part ? e1.z : e1.x;
            const uint32_t b0 = part ? e0.w : e0.y, b1 = part ? e1.w : e1.y;
            ch[0][0][k] = prmt(a0, a1, 0x5410);
            ch[1][0][k] = prmt(a0, a1, 0x7632);
            ch[2][0][k] = prmt(b0, b1, 0x5410);
            ch[3][0][k] = prmt(b0, b1, 0x7632);
          } else {
            ch[0][0][k] = prmt(e0.x, e1.x, 0x5410);
            ch[1][0][k] = prmt(e0.x, e1.x, 0x7632);
            ch[2][0][k] = prmt(e0.y, e1.y, 0x5410);
            ch[3][0][k] = prmt(e0.y, e1.y, 0x7632);
            ch[0][kA1Parts - 1][k] = prmt(e0.z, e1.z, 0x5410);
            ch[1][kA1Parts - 1][k] = prmt(e0.z, e1.z, 0x7632);
            ch[2][kA1Parts - 1][k] = prmt(e0.w, e1.w, 0x5410);
            ch[3][kA1Parts - 1][k] = prmt(e0.w, e1.w, 0x7632);
          }
        } else {
          const uint2 e0 = *reinterpret_cast<const uint2 *>(tb16 + po[uu][2 * k]);
          const uint2 e1 = *reinterpret_cast<const uint2 *>(tb16 + po[uu][2 * k + 1]);
          ch[0][0][k] = prmt(e0.x, e1.x, 0x5410);
          ch[1][0][k] = prmt(e0.x, e1.x, 0x7632);
          ch[2][0][k] = prmt(e0.y, e1.y, 0x5410);
          ch[3][0][k] = prmt(e0.y, e1.y, 0x7632);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < kA1Parts; ++p) {
          const uint32_t ta = tmem + lane_base + kA1 + (uint32_t)((c * kA1Parts + p) * kA1Stride + 4 * u);
          tmem_st_x4(ta, ch[c][p][0], ch[c][p][1], ch[c][p][2], ch[c][p][3]);
        }
    }
    tmem_st_wait();
  };

  // ---- row MMAs: issuer warp 16 + c issues channel c into D1[32 c ..].
  auto issue_row = [&](int part) {
    const int c0 = iw;
    const uint64_t br_desc = smem_desc(smem_u32(BR), 128, 256);
    constexpr uint32_t idesc = idesc_f16(128, 32, BF, 0, 0);
#pragma unroll
    for (int i = 0; i < KXC; ++i) {
      if (i < kcr) {
#pragma unroll
        for (int pp = 0; pp < NSPLIT; ++pp)
#pragma unroll
          for (int cc = 0; cc < 1; ++cc) {
            // products: (data hi, w hi), (data lo, w hi), (data hi, w lo)
            const int c = c0 + cc, ap = pp == 1 ? 1 : 0, bp = pp == 2 ? 1 : 0;
            if (SEQ && ap != part) continue;  // SEQ: A1 holds data part `part` only
            const uint32_t region = SEQ ? (uint32_t)c : (uint32_t)(c * kParts + ap);
            const bool first = i == 0 && (SEQ ? (part == 0 && pp == 0) : pp == 0);
            mma_ts(tmem + kD1 + (uint32_t)(32 * c), tmem + kA1 + region * kA1Stride + (uint32_t)(8 * i),
                   br_desc + (uint64_t)(((i * kWParts + bp) * 1024) >> 4), idesc, first ? 0u : 1u);
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
  // [8h, 8h + 8) x slots (G_r, F_r, G_i, F_i), d_n already folded in; (cos,
  // sin)(n w f) of the demodulation unit from the 2T-phase table, whose offsets
  // then advance to n + 1.
  float P[8], Q[8];
  auto demod = [&](int n) {
    uint32_t v[32];
    tmem_ld_x16(tmem + lane_base + kD2 + (uint32_t)(32 * h), *reinterpret_cast<uint32_t(*)[16]>(&v[0]));
    tmem_ld_x16(tmem + lane_base + kD2 + (uint32_t)(32 * h + 16), *reinterpret_cast<uint32_t(*)[16]>(&v[16]));
    float2 cs[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cs[j] = *reinterpret_cast<const float2 *>(trig + tb + mo[j]);
      mo[j] = wrap(mo[j] + (int)((j & 1) ? (vo[j >> 1] >> 16) : (vo[j >> 1] & 0xFFFFu)));
    }
    tmem_ld_wait_dep(*reinterpret_cast<uint32_t(*)[16]>(&v[0]));
    tmem_ld_wait_dep(*reinterpret_cast<uint32_t(*)[16]>(&v[16]));
    const float dn = kFold ? 1.f : A->d[n];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float tc = dn * cs[j].x, ts = dn * cs[j].y;
      Q[j] = fmaf(tc, __uint_as_float(v[4 * j + 0]), fmaf(ts, __uint_as_float(v[4 * j + 2]), Q[j]));
      P[j] = fmaf(tc, __uint_as_float(v[4 * j + 1]), fmaf(ts, __uint_as_float(v[4 * j + 3]), P[j]));
    }
  };

  // End of the CTA (each role calls it once, after its loop): when a bounded
  // wait gave up, let this CTA's MMAs and TMA copy in flight land (full limit)
  // and record the failure; then release the TMEM.
  auto finish = [&](bool ok) {
    if (!ok) {
      if (col_issuer || row_issuer) mma_commit(mbarD);
      mbar_wait_suspend(mbarD, 0, kDrainPolls, kWaitHintNs);
      if (tma_pending) mbar_wait_suspend(mbarT, phT, kDrainPolls, kWaitHintNs);
      if (tid == 0) atomicOr(x.err, (unsigned)(tmem_ok ? kErrTimeout : kErrTmem));
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(*tmem_base_s, 512);
  };

  // Issuing warpgroup: the same sequence of CTA barriers as the compute loop
  // below, issuing at each point what the barrier made ready.
  bool ok = tmem_ok;
  if (!compute) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(BATCH || kNoA ? kRegIssueBatch : kRegIssue));
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      int K = A->K;
      if (BATCH) {  // this item's image: its harmonics and row chunks
        const FilterArgs *p = bt.imgs + item_image(it);
        K = p->K;
        kcr = kx_of(p->W) / 16;
      }
      if (item_tma(it)) {
        if (mbar_wait_bounded(mbarT, phT, polls)) {
          phT ^= 1;
          tma_pending = false;
        } else {
          fail = true;
        }
        if (!phase_sync()) {
          ok = false;
          break;
        }
      }
      if (!phase_sync()) {  // the compute warps have read the box (and set up a new image)
        ok = false;
        break;
      }
      const int nx = it + (int)gridDim.x;
      if (nx < nitems && item_tma(nx)) {
        if (tma_issuer) issue_tma(nx);
        tma_pending = true;
      }
      if (!(ok = phase_sync())) break;  // table of harmonic 0
      if (!(ok = phase_sync())) break;  // A1 <- harmonic 0 (SEQ: its hi part)
      if (row_issuer) issue_row(0);     // R(0) (SEQ: hi part)
      if (SEQ) {
        if (!(ok = phase_sync())) break;  // A1 <- lo part
        if (row_issuer) issue_row(1);
      }
      if (!(ok = phase_sync())) break;  // B2 <- harmonic 0
      for (int n = 0; n < K; ++n) {
        const bool more = n + 1 < K;
        if (col_issuer) issue_col();  // C(n)
        if (!kNoA && !(ok = phase_sync())) break;  // A1 <- harmonic n + 1 (SEQ: hi part)
        if (SHARED) {
          if (!(ok = phase_sync())) break;  // D2 (= D1) read
          if (more && row_issuer) issue_row(0);
          if (SEQ && more) {
            if (!(ok = phase_sync())) break;  // A1 <- lo part
            if (row_issuer) issue_row(1);
          }
        } else if (more && row_issuer) {  // R(n+1) (kNoA: once every compute warp has stored A1)
          if (!kNoA) {
            issue_row(0);
          } else if (mbar_wait_bounded(mbarA, phA, polls)) {
            fence_after_sync();
            issue_row(0);
            phA ^= 1;
          } else {
            fail = true;
            phA ^= 1;
          }
        }
        if (!(ok = phase_sync())) break;  // B2 <- harmonic n + 1
      }
    }
    finish(ok);
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegCompute));
    int cur = -1;       // batch: image whose tables are set up
    float cur_T = -1.f; // batch: T of the 2T-phase table
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int t = item_tile(it);
      const bool tma_here = item_tma(it);
      if (tma_here) {
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
      if (BATCH) {
        const int img = item_image(it);
        // the image's scalars are read again for every tile (L1 hits) instead
        // of being held in registers across the harmonic loop (with them held,
        // the 6- and 8-chunk batched instantiations spilled)
        set_image(bt.imgs + img);
        if (img != cur) {  // another image: its tables (no MMA is in flight between tiles)
          cur = img;
          if (A->T != cur_T) {
            setup_trig(tid, kNC);
            cur_T = A->T;
          }
          setup_row_toeplitz(tid, kNC);
          if (tmem_ok) setup_col_toeplitz();
        }
      }
      const int ty = t / A->tiles_x;
      const int ty0 = ty * BYv, tx0 = (t - ty * A->tiles_x) * kBX;
      const int iy = ty0 - W + r;  // image row of this thread's ext row
      // ---- load the thread's pixels: REFLECT mirrors (repeatedly, for windows
      // wider than the image); TRUNCATE marks pixels outside the image, whose
      // channels are zero (the zero table entries, no phase step).
      {
        const int bx0 = box_x0(tx0, Wp), by0 = ty0 - W;
        bool row_in = iy >= 0 && iy < H;
        const int sy = reflect ? reflect_index(iy, H) : iy;
        const unsigned char *in = static_cast<const unsigned char *>(A->in);
        const size_t in_pitch = A->in_pitch;
        const float inv2T = 1.0f / (float)twoT;
  #pragma unroll
        for (int uu = 0; uu < UPT; ++uu) {
          const int u = uu == 0 ? demod_u : halo_unit(uu - 1);
          int vm[8];
          // A unit whose 8 pixels lie inside the image and the box (the common
          // case) is one aligned 8-byte read of the box: the box starts at a
          // multiple of 16 columns below tx0 - Wp, and units start at multiples
          // of 8 from there.
          const int ix0 = tx0 - Wp + 8 * (u < 0 ? 0 : u);
          const int ry = (reflect ? sy : iy) - by0, bxu = ix0 - bx0;
          const bool fast = tma_here && u >= 0 && (reflect || row_in) && ix0 >= 0 && ix0 + 8 <= Wd && ry >= 0 &&
                            ry < kLanes && bxu >= 0 && bxu + 8 <= kBoxW;
          uint2 w8 = make_uint2(0u, 0u);
          if (fast) w8 = *reinterpret_cast<const uint2 *>(box + ry * kBoxW + bxu);
  #pragma unroll
          for (int j = 0; j < 8; ++j) {
            int v = 0;
            bool valid = true;
            if (fast) {
              v = (int)(((j < 4 ? w8.x : w8.y) >> (8 * (j & 3))) & 0xFFu);
            } else {
              const int ix = ix0 + j;
              bool in_img = row_in && ix >= 0 && ix < Wd;
              int sx = ix;
              if (reflect) {
                sx = reflect_index(ix, Wd);
                in_img = true;
              }
              if (in_img && u >= 0) {
                const int by = (reflect ? sy : iy) - by0, bx = sx - bx0;
                if (tma_here && by >= 0 && by < kLanes && bx >= 0 && bx < kBoxW)
                  v = box[by * kBoxW + bx];
                else
                  v = __ldg(in + (size_t)(reflect ? sy : iy) * in_pitch + sx);
              }
              valid = in_img && u >= 0;
            }
            po[uu][j] = (valid ? v : kZeroV) * kEntry + copy_off;
            if (uu == 0) {
              mo[j] = valid ? copy8 : copy8 - kCopies * 8;  // entry m = 0, or the zero entry
              // (the batched instantiation keeps the integer form: with the
              // reciprocal it ran 3% slower on the 64-image batch, measured)
              vm[j] = valid ? (BATCH ? (v < twoT ? v : v % twoT) : mod2T(v, inv2T)) * (kCopies * 8) : 0;
            }
          }
          if (uu == 0) {
  #pragma unroll
            for (int k = 0; k < 4; ++k) vo[k] = (uint32_t)vm[2 * k] | ((uint32_t)vm[2 * k + 1] << 16);
          }
        }
      }
      // every thread has read the box: the next tile's copy may overwrite it
      // (and a new image's row Toeplitz blocks are visible to the MMAs)
      fence_proxy_async_smem();
      if (!phase_sync()) {
        ok = false;
        break;
      }
      const int nx = it + (int)gridDim.x;
      if (nx < nitems && item_tma(nx)) tma_pending = true;
  #pragma unroll
      for (int j = 0; j < 8; ++j) P[j] = Q[j] = 0.f;
      const int K = A->K;

      // ---- prologue: the tables of harmonics 0 and 1; harmonic 0 through the row
      // pass and the re-split.  The table of harmonic n is in buffer n % 2.
      bm = 0;
      build_table(0, 0);
      if (!(ok = phase_sync())) break;
      modulate(0, 0);
      if (!(ok = phase_sync())) break;
      if (K > 1) build_table(1, 1);
      wait_bar(mbarR, phR);
      if (SEQ) {  // the lo part through the same A1
        modulate(0, 1);
        if (!(ok = phase_sync())) break;
        wait_bar(mbarR, phR);
      }
      resplit();
      if (!(ok = phase_sync())) break;

      for (int n = 0; n < K; ++n) {
        const bool more = n + 1 < K;
        if (more) modulate((n + 1) & 1, 0);  // A1 <- harmonic n + 1 (while C(n): B2 -> D2 runs)
        if (!kNoA) {
          if (!(ok = phase_sync())) break;
        } else if (more) {  // this warp's A1 stores are complete: the row MMAs may start
          fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(mbarA);
        }
        // the table of n + 2 replaces that of n (read by the modulation of n, done)
        if (SHARED) {
          if (n + 2 < K) build_table(n + 2, n & 1);
          wait_bar(mbarC, phC);
          demod(n);
          if (!(ok = phase_sync())) break;
          if (more) {  // R(n+1): A1 -> D (= D2, read)
            wait_bar(mbarR, phR);
            if (SEQ) {  // then the lo part of harmonic n + 1 through the same A1
              modulate((n + 1) & 1, 1);
              if (!(ok = phase_sync())) break;
              wait_bar(mbarR, phR);
            }
            resplit();
          }
        } else {
          // R(n+1): A1 -> D1 runs meanwhile
          if (n + 2 < K) build_table(n + 2, n & 1);
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

      // ---- fhat = P / Q + c0, staged in B2 (free: every thread has seen the last
      // column MMAs complete) so that the stores leave as whole 128-byte row
      // segments.  Stage row r = ext row r, 32 floats in eight 16-byte slots,
      // slot s stored at s ^ (r & 7) (conflict-free writes of a warp's 32 rows).
      {
        float *stage = reinterpret_cast<float *>(B2);
  #pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int sl = (2 * h + k) ^ (r & 7);
          *reinterpret_cast<float4 *>(stage + r * 32 + sl * 4) =
              make_float4(P[4 * k] / Q[4 * k] + c0, P[4 * k + 1] / Q[4 * k + 1] + c0, P[4 * k + 2] / Q[4 * k + 2] + c0,
                          P[4 * k + 3] / Q[4 * k + 3] + c0);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kNC) : "memory");  // the compute threads only
        float *out = static_cast<float *>(A->out);
        const size_t opitch = A->out_pitch;
        const bool vec = ((reinterpret_cast<uintptr_t>(out) | opitch) & 15) == 0;
  #pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int e = tid + k * kNC, row = e >> 3, sl = e & 7;  // 128 rows x 8 slots
          const int oy = ty0 - W + row, ox = tx0 + 4 * sl;
          if (row >= W && row < kLanes - W && oy < H && ox < Wd) {
            const float4 v = *reinterpret_cast<const float4 *>(stage + row * 32 + ((sl ^ (row & 7)) * 4));
            float *orow = reinterpret_cast<float *>(reinterpret_cast<char *>(out) + (size_t)oy * opitch);
            if (vec && ox + 4 <= Wd) {
              *reinterpret_cast<float4 *>(orow + ox) = v;
            } else {
              orow[ox] = v.x;
              if (ox + 1 < Wd) orow[ox + 1] = v.y;
              if (ox + 2 < Wd) orow[ox + 2] = v.z;
              if (ox + 3 < Wd) orow[ox + 3] = v.w;
            }
          }
        }
      }
    }
    finish(ok);
  }
}

// One image (the single-image entry points).
template <int BF, int NSPLIT, int KXC, int SHARED, int SEQ = 0>
__global__ void __launch_bounds__(kNT, 1) fbf_tc2_u8_kernel(const __grid_constant__ FilterArgs a,
                                                             const __grid_constant__ CUtensorMap tmap,
                                                             const Tc2Extra x) {
  const Tc2Batch none{};
  tc2_body<BF, NSPLIT, KXC, SHARED, SEQ, false>(&a, &tmap, none, x);
}

// A batch of images in one persistent launch (batched plans).
template <int BF, int NSPLIT, int KXC, int SHARED, int SEQ = 0>
__global__ void __launch_bounds__(kNT, 1) fbf_tc2_batched_kernel(const __grid_constant__ Tc2Batch b,
                                                                  const Tc2Extra x) {
  tc2_body<BF, NSPLIT, KXC, SHARED, SEQ, true>(nullptr, nullptr, b, x);
}

}  // namespace tc2
}  // namespace fbf

namespace fbf {
namespace tc2 {

// Host launcher of one instantiation: tiles of 32 x (128 - 2W), one persistent
// CTA per SM (at most one per tile), the box tensor map from the per-pointer
// cache, the shared-memory attribute set once per device.
template <int BF, int NSPLIT, int KXC, int SHARED, int SEQ = 0>
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
  auto kern = fbf_tc2_u8_kernel<BF, NSPLIT, KXC, SHARED, SEQ>;
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

// Host launcher of a batch (device tables prepared by the caller, every image
// within the instantiation's window): one persistent CTA per SM, at most one
// per item.
template <int BF, int NSPLIT, int KXC, int SHARED, int SEQ = 0>
fbf_status launch_batch_cfg(const Tc2Batch &b, cudaStream_t s) {
  if (b.nitems <= 0) return FBF_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FBF_ERR_CUDA;
  const int sms = sm_count(dev);
  if (sms <= 0) return FBF_ERR_CUDA;
  const int grid = b.nitems < sms ? b.nitems : sms;
  constexpr Layout Ly = layout<NSPLIT, KXC>();
  auto kern = fbf_tc2_batched_kernel<BF, NSPLIT, KXC, SHARED, SEQ>;
  static FuncAttrOnce once;
  if (!once.done(dev)) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Ly.bytes) != cudaSuccess)
      return FBF_ERR_CUDA;
    once.set(dev);
  }
  Tc2Extra x{device_error_word(), wait_polls(), 0};
  if (!x.err) return FBF_ERR_CUDA;
  kern<<<grid, kNT, Ly.bytes, s>>>(b, x);
  return cuda_status(cudaGetLastError());
}

}  // namespace tc2
}  // namespace fbf
