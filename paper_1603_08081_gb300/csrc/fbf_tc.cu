// Tensor-core form of the fused shiftable bilateral filter (Algorithm 1) for
// uint8 images: both 1-D passes of every harmonic run as banded-Toeplitz
// products on the 5th-generation tensor cores (tcgen05.mma, kind::f16, FP32
// accumulation in tensor memory).
//
// One CTA (512 threads: four groups of four warps, warp w reaching TMEM lanes
// 32 (w % 4) ... + 31) owns a tile of 32 output columns and min(BY, 128 - 2W)
// output rows, whose halo rows fill at most the 128 TMEM lanes (BY = 112
// computed rows for W <= 16, 96 for W <= 26, 64 for W <= 32; rows computed
// past 128 - 2W have a clipped band and are discarded).  Taller tiles mean
// fewer tiles: a 2048^2 image at W = 9 is 19 x 64 tiles of 110 rows, 8 waves
// of 152 CTAs, where 96-row tiles took 10.  For each harmonic n:
//
//   modulate  thread (lane r, group h) gathers, for ext row r and its share
//             of the ext columns, the per-harmonic table entry of each pixel
//             value: (cos, sin, f cos, f sin)(n w f) already rounded to 16
//             bits (hi, and lo = the rounding residual for the split forms),
//             pairs neighbouring columns with byte permutes and writes them
//             with tcgen05.st into TMEM: A1[c][part] (lane = ext row, K = ext
//             column, two 16-bit elements per 32-bit column);
//   row MMA   D1[c] (lane = ext row, 32 columns = outputs x) = sum over
//             16-wide K chunks of A1[c][part] * T_i; T_i is the 16 x 32
//             Toeplitz block of chunk offset i (entries w[16 i + k - n]);
//             only the ceil((32 + 2W) / 16) chunks that meet the band are
//             issued;
//   re-split  D1 rows are read back (tcgen05.ld), rounded to 16 bits again
//             (hi, lo) and stored to shared memory as the MN-major A operand
//             of the column pass, A2[m = 4 x + c][K = ext row] -- each thread
//             writes its own row, so no transpose is needed;
//   col MMA   D2 (lane m = 4 x + c, columns = output rows y) = sum A2 * T_i,
//             in one output block of BY rows (BY = 112, 96) or, for BY = 64,
//             one of 64 (single form) or two of 32 (split forms); wide
//             blocks take their Toeplitz blocks as windows of one shared strip;
//   demod     lane (c, x) accumulates d_n * trig(n w f(y, x)) * D2 into its
//             own partial: cos for the G_r / F_r channels, sin for G_i / F_i.
//
// P = partial(F_r) + partial(F_i), Q = partial(G_r) + partial(G_i) are combined
// once per tile, and fhat = P / Q + c0 is written.  The f channels carry
// (f - c0) with c0 = T / 2 instead of f: the sums become P - c0 Q, the ratio is
// unchanged in exact arithmetic, and the magnitudes rounded to 16 bits halve.
//
// Schedule (pipelined; the serial one for the split forms at W > 16): per
// harmonic two phases separated by CTA barriers --
//   (1) group 0 issues the column MMAs of n while groups 1-3 modulate n + 1;
//   (2) group 0 issues the row MMAs of n + 1 while groups 2-3 build the tables
//       of n + 2; then every thread waits for the column MMAs of n (its own
//       mbarrier wait: it reads only its own TMEM lanes), demodulates n, waits
//       for the row MMAs of n + 1 and re-splits them.
// MMAs are issued by lane 0 of the four warps of group 0, which own disjoint
// accumulators; a bounded mbarrier wait that gives up is OR-reduced at the
// next barrier and the CTA stops with a device error word set.
//
// The kernel is persistent (one CTA per SM walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; TMEM, barriers and Toeplitz blocks are set up
// once).  While a tile is processed, the next tile's halo is prefetched by a
// 2-D TMA copy (cp.async.bulk.tensor) into a raw shared-memory box, which the
// next tile converts into the staged tile.  Under TRUNCATE out-of-image box
// entries become the zero-channel sentinel by their coordinates; under REFLECT
// the halo pixels outside the image read their mirrored source inside the box
// (a single mirror reaches it when W < H and W < Wd; otherwise, and for
// unaligned images, the tiles load directly with reflected indices).
//
// Precision: the split forms carry data as hi + lo; FP16 uses one weight part
// (2 products per step), BF16 splits the weights too (3 products); the single
// FP16 form rounds data and weights once (1 product per step: half the MMAs,
// table entries and re-split stores).  Table entries, the phase (exact integer
// reduction), the K-term accumulation and the ratio stay in FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "fbf_common.cuh"
#include "fbf_internal.h"
#include "fbf_tc_ptx.cuh"

__device__ unsigned int g_fbf_tc_error = 0;

namespace fbf {
namespace {

using namespace tc;

constexpr int kCopies = 8;
constexpr int kLutEntries = 257;
constexpr int kSentinel = 256;
constexpr int kLutStride = kLutEntries * kCopies;  // entries per table buffer
// Per harmonic and pixel value v two tables, 8 interleaved copies each:
//   lut16[v]: uint4 of 16-bit (hi c | hi s<<16, hi fc | hi fs<<16, lo c | lo s<<16, lo fc | lo fs<<16)
//   lutf[v]:  float2 (cos, sin) in FP32 for the demodulation.
// The staged tile holds v * 128, the byte offset of v's row in lut16 (half of it in lutf).
constexpr int kBX = 32;                             // output columns per tile
constexpr int kLanes = 128;                         // TMEM lanes = halo rows per tile
// Staged tile, in one of two layouts:
//  * column-major (windows up to 16): one column of 128 ext rows per ext
//    column, pitch kPT u16 (kPT / 2 odd); the modulation reads one u16 per
//    lane and ext column, conflict-free across the lanes (rows).
//  * row-major (wider windows, 3x the ext columns): one row of KX u16 offsets
//    per ext row, padded to a pitch of KXmax + 8 u16 (an odd number of 16-byte
//    units), so that the 16-byte loads of 8 ext columns by neighbouring rows are
//    conflict-free: half the load wavefronts of the column-major reads, at the
//    cost of unpacking the offsets (which costs more than it saves when the
//    tile has few ext columns).
constexpr int kPT = kLanes + 2;
__host__ __device__ constexpr int tile_pitch(int kxmax) { return kxmax + 8; }
__host__ __device__ constexpr bool tile_row_major(int wcap) { return wcap > 16; }
constexpr int kA2Group = 2048;                      // bytes per 8-row K group of A2 (16 M groups x 128 B)
constexpr int kA2Part = 16 * kA2Group;              // one part of A2: 128 (M) x 128 (K) x 16 bit
constexpr uint32_t kMaxPolls = 1u << 22;

// Output rows of one tile: the BY computed rows, at most the kLanes - 2W rows
// whose 2W + 1 taps all lie in the 128 ext rows (the rows past that are
// computed with a truncated band and discarded).
__host__ __device__ __forceinline__ constexpr int tile_rows(int by, int W) { return by < kLanes - 2 * W ? by : kLanes - 2 * W; }
// Column pass: output blocks of nbc rows (the last one by - (blocks - 1) nbc
// rows).  K chunks of the block of n outputs starting at row `start`: those
// meeting its band, clipped to the 128 ext rows (outputs whose band is clipped
// lie past tile_rows and are discarded).
__host__ __device__ __forceinline__ constexpr int col_chunks(int W, int start, int n) {
  return (n + 2 * W + 15) / 16 < (kLanes - start) / 16 ? (n + 2 * W + 15) / 16 : (kLanes - start) / 16;
}
// The column pass's Toeplitz weights: a strip shared by all K chunks and
// blocks when the blocks are uneven or wide (per-chunk blocks would hold kcc
// blocks of nbc rows), one block per chunk otherwise.  Bytes of one part (sized
// for the widest window):
__host__ __device__ constexpr bool col_strip(int by, int nbc) { return by % nbc != 0 || nbc >= 64; }
__host__ __device__ constexpr int col_b_part(int wcap, int by, int nbc) {
  return col_strip(by, nbc) ? (nbc + 16 * (col_chunks(wcap, 0, nbc) - 1)) * 32
                            : ((nbc + 2 * wcap + 15) / 16) * nbc * 32;
}

struct TcLayout {
  int kcr;  // 16-wide K chunks meeting the band of one NBR-output block (row pass)
  int kcc;  // the same for the first NBC-output block (column pass), clipped to the 128 ext rows
  int KX;   // K extent of the row pass (ext columns, multiple of 16)
  int A1C;  // TMEM columns per (channel, part) of A1 = KX / 2
  size_t lut16_off, lutf_off, a2_off, br_off, bc_off, tile_off, raw_off, trig_off, bar_off, bytes;
};

// (cos, sin)(pi m / T) for the phase indices m < 2T, built once per CTA when
// 2T <= kTrigMax (the per-harmonic tables then look the phase up instead of
// evaluating sincospi on their critical path).
constexpr int kTrigMax = 1024;

constexpr int kBoxW = 112;  // TMA box: 112 columns (>= 15 + KX) x 128 rows of bytes

// Shared memory: [lut16 (one buffer)][lutf (three buffers)][A2 hi | lo]
// [row Toeplitz blocks][column Toeplitz strip][tile][TMA box][trig][barriers, TMEM address, flags].
__host__ __device__ __forceinline__ TcLayout tc_layout(int W, int wcap, int by, int nbr, int nbc) {
  TcLayout L;
  L.kcr = (nbr + 2 * W + 15) / 16;
  L.kcc = col_chunks(W, 0, nbc);
  L.KX = kBX - nbr + 16 * L.kcr;
  L.A1C = L.KX / 2;
  const int kcr_max = (nbr + 2 * wcap + 15) / 16;
  const int KXmax = kBX - nbr + 16 * kcr_max;
  L.lut16_off = 0;
  L.lutf_off = L.lut16_off + (size_t)kLutStride * sizeof(uint4);
  L.a2_off = (L.lutf_off + 3ull * kLutStride * sizeof(float2) + 1023) & ~(size_t)1023;
  L.br_off = L.a2_off + 2ull * kA2Part;
  L.bc_off = L.br_off + (size_t)kcr_max * 2 * nbr * 32;
  L.tile_off = L.bc_off + 2ull * col_b_part(wcap, by, nbc);  // 32-byte aligned
  const size_t tile_bytes =
      tile_row_major(wcap) ? (size_t)kLanes * tile_pitch(KXmax) * 2 : (size_t)KXmax * kPT * 2;
  L.raw_off = (L.tile_off + tile_bytes + 1023) & ~(size_t)1023;  // TMA destination
  L.trig_off = L.raw_off + (size_t)kBoxW * kLanes;
  L.bar_off = L.trig_off + (size_t)kTrigMax * sizeof(float2);
  L.bytes = L.bar_off + 64;
  return L;
}

// Two floats -> packed 16-bit pair (first in the low half) plus the residuals.
template <int BF>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
  if (BF) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
  }
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

// Per-harmonic tables (see above); copies written rotated so that the stores of
// neighbouring values land in different bank groups.  SINGLE: the 16-bit table
// keeps only the hi words (uint2), in 16 copies of 8 bytes (the same 128 bytes
// per value), so that the modulation's 8-byte gathers are conflict-free too.
template <int BF, int NT, int SINGLE>
__device__ __forceinline__ void build_lut(uint4 *L16, float2 *Lf, const float2 *trig, int n, int twoT, float T,
                                          float c0, int tid) {
  for (int v = tid; v < 256; v += NT) {
    const int m = (n * v) % twoT;  // exact phase index: n*omega*v = pi * m / T (mod 2 pi)
    float sn, cs;
    if (twoT <= kTrigMax) {
      const float2 t = trig[m];
      cs = t.x;
      sn = t.y;
    } else {
      sincospif((float)m / T, &sn, &cs);
    }
    const float fv = (float)v - c0;  // centred intensity
    uint4 e;
    split2<BF>(cs, sn, e.x, e.z);
    split2<BF>(fv * cs, fv * sn, e.y, e.w);
    const float2 f = make_float2(cs, sn);
    if (SINGLE) {
      uint2 *L8 = reinterpret_cast<uint2 *>(L16);
#pragma unroll
      for (int j = 0; j < 2 * kCopies; ++j) L8[v * 2 * kCopies + ((j + v) & (2 * kCopies - 1))] = make_uint2(e.x, e.y);
    } else {
#pragma unroll
      for (int j = 0; j < kCopies; ++j) L16[v * kCopies + ((j + v) & (kCopies - 1))] = e;
    }
#pragma unroll
    for (int j = 0; j < kCopies; ++j) Lf[v * kCopies + ((j + (v >> 1)) & (kCopies - 1))] = f;
  }
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Toeplitz strip of the column pass: the K chunk i block of an output block,
// B_i(n, k) = w[16 i + k - n], equals S(n - 16 i, k) with S(r, k) = w[k - r]
// inside the band and 0 outside, so one strip of the NB + 16 (kc - 1) rows
// r = -16 (kc - 1) ... NB - 1 (same K-major layout, row r at index r + 16 (kc - 1))
// serves every chunk i < kc of every block of up to NB outputs: chunk i's
// descriptor starts 2 (kc - 1 - i) 8-row groups in.
// Part 0 holds the 16-bit weights, part 1 (part_bytes further) their residuals.
template <int BF, int NB, int NT>
__device__ __forceinline__ void build_toeplitz_strip(unsigned char *B, int kc, int part_bytes, int W, const float *w,
                                                     int tid) {
  const int rows = NB + 16 * (kc - 1);
  for (int e = tid; e < rows * 16; e += NT) {
    const int n = e >> 4, k = e & 15;  // strip row n = r + 16 (kc - 1)
    const int t = k - (n - 16 * (kc - 1));
    const float wv = (t >= 0 && t <= 2 * W) ? w[t] : 0.f;
    const unsigned short hi = to16<BF>(wv);
    const unsigned short lo = to16<BF>(wv - from16<BF>(hi));
    const int off = (n & 7) * 16 + (n >> 3) * 256 + (k & 7) * 2 + (k >> 3) * 128;
    *reinterpret_cast<unsigned short *>(B + off) = hi;
    *reinterpret_cast<unsigned short *>(B + part_bytes + off) = lo;
  }
}

// Toeplitz blocks for output blocks of NB: block i (K chunk offset i) holds
// element (n, k) = w[16 i + k - n] inside the band and 0 outside, K-major
// without swizzle ((n % 8) * 16 + (n / 8) * 256 + (k % 8) * 2 + (k / 8) * 128);
// part 0 is the 16-bit weight, part 1 its residual.
template <int BF, int NB, int NT>
__device__ __forceinline__ void build_toeplitz(unsigned char *B, int nblocks, int W, const float *w, int tid) {
  for (int e = tid; e < nblocks * NB * 16; e += NT) {
    const int i = e / (NB * 16), rem = e - i * NB * 16, n = rem >> 4, k = rem & 15;
    const int t = 16 * i + k - n;
    const float wv = (t >= 0 && t <= 2 * W) ? w[t] : 0.f;
    const unsigned short hi = to16<BF>(wv);
    const unsigned short lo = to16<BF>(wv - from16<BF>(hi));
    const int off = (n & 7) * 16 + (n >> 3) * 256 + (k & 7) * 2 + (k >> 3) * 128;
    *reinterpret_cast<unsigned short *>(B + (size_t)(2 * i) * NB * 32 + off) = hi;
    *reinterpret_cast<unsigned short *>(B + (size_t)(2 * i + 1) * NB * 32 + off) = lo;
  }
}

// BF: 0 = FP16, 1 = BF16.  NSPLIT: 1 = data hi x weights hi; 2 = data hi/lo x
// weights hi; 3 = plus data hi x weights lo.
// BY: output rows per tile (BY + 2 * WCAP <= 128).  NBR / NBC: MMA N (output
// block) of the row / column pass; bigger blocks issue fewer, larger MMAs at the
// price of more zero taps inside each block.  NT: threads (256 or 512); the
// NT / 32 warps form NT / 128 groups of four, each group covering the 128 TMEM
// lanes once (warp w reaches lanes 32 (w % 4) ... + 31).
template <int BF, int NSPLIT, int BY, int WCAP, int NBR, int NBC, int PIPE, int NT>
__global__ void __launch_bounds__(NT, 1) fbf_tc_u8_kernel(const __grid_constant__ FilterArgs a,
                                                           const __grid_constant__ CUtensorMap tmap, int use_tma) {
  // Computed rows: BY (multiple of 16, up to 128); the demodulation reads the
  // centre pixels of rows W ... W + BY - 1 of the 128 staged ext rows.
  static_assert(BY <= kLanes && BY % 16 == 0 && BY + WCAP <= kLanes, "computed rows fit the TMEM lanes");
  static_assert(tile_rows(BY, WCAP) >= 32, "output rows per tile");
  static_assert(kBX % NBR == 0 && NBR % 16 == 0 && NBC % 16 == 0 && NBC <= 256, "output blocks");
  static_assert(NSPLIT >= 1 && NSPLIT <= 3, "products per step");
  constexpr int kParts = NSPLIT > 1 ? 2 : 1;  // data parts held in A1 / A2 (hi, lo)
  // A1 (4 kParts regions of KX/2 columns) must fit below D1: 256 columns when
  // pipelined (D1 at 256, D2 at 384), 384 otherwise (D1 at 384, D2 over A1).
  static_assert(2 * kParts * (kBX - NBR + 16 * ((NBR + 2 * WCAP + 15) / 16)) <= (PIPE ? 256 : 384),
                "A1 fits below D1");
  static_assert(NT == 256 || NT == 512, "two or four warp groups");
  constexpr int kGroups = NT / 128;   // warp groups; h = warp / 4 in [0, kGroups)
  constexpr int BYH = BY / kGroups;   // output rows per thread in the demodulation
  constexpr int XPT = kBX / kGroups;  // outputs x per thread in the re-split
  static_assert(BYH % 4 == 0 && XPT % 8 == 0, "TMEM loads in groups of 4 / 8 columns");
  static_assert(4 * (BY * kBX + 8) * 4 <= 2 * kA2Part, "combine planes fit the A2 region");
  static_assert((PIPE ? 384 : 0) + BY <= 512, "D2 fits the TMEM columns");
  constexpr int NP = NSPLIT;   // products per (chunk, output block)
  // MMAs are issued by lane 0 of several warps (a single issuing thread would
  // spend ~50 cycles per small MMA); every issuer owns whole accumulator blocks.
  constexpr int kRowIssuers = 4;                                 // one per channel
  constexpr int kColBlocks = (BY + NBC - 1) / NBC;
  constexpr int kLastN = BY - (kColBlocks - 1) * NBC;  // outputs of the last column block
  constexpr bool kStrip = col_strip(BY, NBC);
  static_assert(kStrip || BY - NBC + 16 * ((NBC + 2 * WCAP + 15) / 16) <= kLanes, "column-pass K fits A2");
  constexpr int kColIssuers = kColBlocks < 4 ? kColBlocks : 4;  // output blocks j = w, w + 4, ...
  extern __shared__ __align__(1024) unsigned char smem[];
  const int W = a.W;
  const TcLayout Ly = tc_layout(W, WCAP, BY, NBR, NBC);
  // output rows of a tile (all BY computed rows when every window up to WCAP allows)
  const int BYv = BY + 2 * WCAP <= kLanes ? BY : tile_rows(BY, W);
  constexpr int kBcPart = col_b_part(WCAP, BY, NBC);
  uint4 *lut16 = reinterpret_cast<uint4 *>(smem + Ly.lut16_off);
  float2 *lutf = reinterpret_cast<float2 *>(smem + Ly.lutf_off);
  unsigned char *A2 = smem + Ly.a2_off;
  unsigned short *tileT = reinterpret_cast<unsigned short *>(smem + Ly.tile_off);
  // element (ext row ey, ext column ex) of the staged tile at ey * kTY + ex * kTX
  constexpr bool kRM = tile_row_major(WCAP);
  constexpr int kTP = tile_pitch(kBX - NBR + 16 * ((NBR + 2 * WCAP + 15) / 16));
  static_assert(!kRM || (kTP * 2 / 16) % 2 == 1, "odd number of 16-byte units per tile row");
  constexpr int kTY = kRM ? kTP : 1, kTX = kRM ? 1 : kPT;
  uint64_t *mbarR = reinterpret_cast<uint64_t *>(smem + Ly.bar_off);      // row MMAs done
  uint64_t *mbarC = reinterpret_cast<uint64_t *>(smem + Ly.bar_off + 8);  // column MMAs done
  uint32_t *tmem_base_s = reinterpret_cast<uint32_t *>(smem + Ly.bar_off + 16);
  int *abort_s = reinterpret_cast<int *>(smem + Ly.bar_off + 32);
  uint64_t *mbarT = reinterpret_cast<uint64_t *>(smem + Ly.bar_off + 40);  // TMA box landed
  unsigned char *raw = smem + Ly.raw_off;
  float2 *trig = reinterpret_cast<float2 *>(smem + Ly.trig_off);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, cp = lane & (kCopies - 1);
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quadrant, warp group
  const int H = a.H, Wd = a.Wd, HY = BYv + 2 * W, HX = kBX + 2 * W;
  const int kcr = Ly.kcr, kcc = kStrip ? Ly.kcc : (NBC + 2 * W + 15) / 16, A1C = Ly.A1C, KX = Ly.KX;
  const bool reflect = a.border == FBF_BORDER_REFLECT;
  const float c0 = 0.5f * a.T;  // intensity centre
  constexpr unsigned short kScale = kCopies * sizeof(uint4), kSent = kSentinel * kCopies * sizeof(uint4);

  // Whether the tiles' halos come through the TMA box: always under TRUNCATE;
  // under REFLECT when a single mirror reaches every halo pixel (W < H, W < Wd):
  // the mirrored source of every halo pixel that can touch an output inside
  // the image (rows < H + W, columns < Wd + W) then lies inside the box.
  const bool tma_all = use_tma && (!reflect || (W < H && W < Wd));
  auto tma_tile = [&](int) -> bool { return tma_all; };
  auto mirror = [](int i, int n) -> int { return i < 0 ? -i - 1 : (i >= n ? 2 * n - 1 - i : i); };
  auto box_x = [&](int t) -> int {  // 16-byte aligned start column of tile t's box
    const int tx = t - (t / a.tiles_x) * a.tiles_x;
    const int x0 = tx * kBX - W;
    return x0 >= 0 ? (x0 & ~15) : -((-x0 + 15) & ~15);
  };
  auto issue_tma = [&](int t) {  // one thread
    const int ty = t / a.tiles_x;
    mbar_arrive_expect_tx(mbarT, (uint32_t)(kBoxW * kLanes));
    tma_load_2d(raw, &tmap, box_x(t), ty * BYv - W, mbarT);
  };

  if (warp == 0) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(mbarR, kRowIssuers);  // one commit per issuing warp
    mbar_init(mbarC, kColIssuers);
    mbar_init(mbarT, 1);
    mbar_fence_init();
    *abort_s = 0;
  }
  if (tid < kCopies) lut16[kSentinel * kCopies + tid] = make_uint4(0u, 0u, 0u, 0u);
  if (tid < 3 * kCopies)  // sentinel rows: zero channels
    lutf[(tid / kCopies) * kLutStride + kSentinel * kCopies + (tid % kCopies)] = make_float2(0.f, 0.f);
  if (a.twoT <= kTrigMax)
    for (int m = tid; m < a.twoT; m += NT) sincospif((float)m / a.T, &trig[m].y, &trig[m].x);
  build_toeplitz<BF, NBR, NT>(smem + Ly.br_off, kcr, W, a.w, tid);
  if constexpr (kStrip)
    build_toeplitz_strip<BF, NBC, NT>(smem + Ly.bc_off, kcc, kBcPart, W, a.w, tid);
  else
    build_toeplitz<BF, NBC, NT>(smem + Ly.bc_off, kcc, W, a.w, tid);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (tid == 0 && blockIdx.x < a.ntiles && tma_tile(blockIdx.x)) issue_tma(blockIdx.x);

  const uint32_t tmem = *tmem_base_s;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  // TMEM column bases: pipelined, A1 | D1 | D2 are disjoint; otherwise D2 reuses A1.
  const uint32_t kA1 = 0, kD1 = PIPE ? 256 : 384, kD2 = PIPE ? 384 : 0;
  constexpr uint32_t idesc_row = idesc_f16(128, NBR, BF, 0, 0);
  constexpr uint32_t idesc_col = idesc_f16(128, NBC, BF, 1, 0);
  constexpr uint32_t idesc_col_last = idesc_f16(128, kLastN, BF, 1, 0);
  // Descriptor bases; offsets below 256 KB are added to the low address field.
  const uint64_t br_desc = smem_desc(smem_u32(smem + Ly.br_off), 128, 256);
  const uint64_t bc_desc = smem_desc(smem_u32(smem + Ly.bc_off), 128, 256);
  const uint64_t a2_desc = smem_desc(smem_u32(A2), kA2Group, 128);
  // Gather base: copy cp of the 8 16-byte entries, or copy lane % 16 of the 16
  // 8-byte entries of the single form.
  const char *L16 = kParts == 2 ? reinterpret_cast<const char *>(lut16 + cp)
                                : reinterpret_cast<const char *>(lut16) + 8 * (lane & (2 * kCopies - 1));

  float part[BYH];
  uint32_t cen_pk[BYH / 2] = {};  // lutf byte offsets of this thread's demodulation pixels, two per register
  auto cen_off = [&](int j) -> uint32_t { return (j & 1) ? (cen_pk[j >> 1] >> 16) : (cen_pk[j >> 1] & 0xFFFFu); };
  uint32_t phR = 0, phC = 0, phT = 0;
  bool ok = true;
  // The FP32 (cos, sin) table of harmonic n of the current tile is buffer
  // (lbase + n) % 3; lbase advances by K per tile, so that in the pipelined
  // schedule the next tile's tables of harmonic 0 are built as harmonic K of
  // this one (in the phase that builds harmonic n + 2), not at its start.
  int lbase = 0;
  bool t0_ready = false;  // the tables of harmonic 0 of the current tile are built
  bool tma_pending = blockIdx.x < a.ntiles && tma_tile(blockIdx.x);  // a box copy is in flight

  // ---- modulate harmonic n: ext row r = 32 q + lane; units of 4 TMEM columns
  // (8 ext columns) u = h, h + kGroups, ... of the A1C / 4 units.
  // With four warp groups, group 0 (whose lane-0 threads issue the MMAs)
  // takes no modulation units and no table building: the issue cost overlaps
  // the other groups' work instead of delaying group 0's share of it.
  constexpr int kModGroups = kGroups > 2 ? kGroups - 1 : kGroups;
  const int hm = kGroups > 2 ? h - 1 : h;                     // -1: no modulation units
  const int btid = kGroups > 2 ? (tid >= 256 ? tid - 256 : 256) : tid;  // table-building index
  auto modulate = [&]() {
    const unsigned short *trow = tileT + (32 * q + lane) * kTY;
#pragma unroll 1
    for (int u = hm; u >= 0 && u < A1C / 4; u += kModGroups) {
      const int col = 4 * u;
      uint32_t ow[4];  // row-major: offsets of ext columns 8u .. 8u + 7, two per word
      if constexpr (kRM) {
        const uint4 o = *reinterpret_cast<const uint4 *>(trow + 8 * u);
        ow[0] = o.x, ow[1] = o.y, ow[2] = o.z, ow[3] = o.w;
      }
      uint4 e[8];  // table entries of 8 ext columns (the single form reads the hi half only)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t off;
        if constexpr (kRM)
          off = (j & 1) ? (ow[j >> 1] >> 16) : (ow[j >> 1] & 0xFFFFu);
        else
          off = trow[(8 * u + j) * kTX];
        if (kParts == 2) {
          e[j] = *reinterpret_cast<const uint4 *>(L16 + off);
        } else {
          const uint2 hi = *reinterpret_cast<const uint2 *>(L16 + off);
          e[j] = make_uint4(hi.x, hi.y, 0u, 0u);
        }
      }
      uint32_t v[8][4];  // [channel * kParts + part][column]
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 a0 = e[2 * j], a1 = e[2 * j + 1];
        v[0 * kParts][j] = prmt(a0.x, a1.x, 0x5410);  // cos hi
        v[1 * kParts][j] = prmt(a0.x, a1.x, 0x7632);  // sin hi
        v[2 * kParts][j] = prmt(a0.y, a1.y, 0x5410);  // f cos hi
        v[3 * kParts][j] = prmt(a0.y, a1.y, 0x7632);  // f sin hi
        if (kParts == 2) {
          v[1][j] = prmt(a0.z, a1.z, 0x5410);  // cos lo
          v[3][j] = prmt(a0.z, a1.z, 0x7632);  // sin lo
          v[5][j] = prmt(a0.w, a1.w, 0x5410);  // f cos lo
          v[7][j] = prmt(a0.w, a1.w, 0x7632);  // f sin lo
        }
      }
#pragma unroll
      for (int cp2 = 0; cp2 < 4 * kParts; ++cp2)
        tmem_st_x4(tmem + lane_base + kA1 + (uint32_t)(cp2 * A1C + col), v[cp2][0], v[cp2][1], v[cp2][2],
                   v[cp2][3]);
    }
    tmem_st_wait();
  };

  // ---- row MMAs: lane 0 of warp c issues channel c (its own accumulators).
  const bool row_issuer = lane == 0 && warp < kRowIssuers;
  const bool col_issuer = lane == 0 && warp < kColIssuers;
  auto issue_row = [&]() {
    fence_after_sync();
    const int c = warp;
#pragma unroll 1
    for (int i = 0; i < kcr; ++i)
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) {
        const int ap = pp == 1 ? 1 : 0;  // data part: hi, lo, hi
        const int bp = pp == 2 ? 1 : 0;  // weight part: hi, hi, lo
        const uint64_t bd = br_desc + (uint64_t)(((2 * i + bp) * NBR * 32) >> 4);
#pragma unroll
        for (int j = 0; j < kBX / NBR; ++j)
          mma_ts(tmem + kD1 + (uint32_t)(c * 32 + j * NBR),
                 tmem + kA1 + (uint32_t)((kParts * c + ap) * A1C + (j * NBR / 16 + i) * 8), bd, idesc_row,
                 (i > 0 || pp > 0) ? 1u : 0u);
      }
    mma_commit(mbarR);
  };

  // ---- re-split the row-pass result into the column pass's A operand.
  // Thread: ext row r, outputs x in [XPT h, XPT h + XPT), all four channels;
  // A2[m = 4 x + c][r] is MN-major:
  // (m % 8) * 2 + (r % 8) * 16 + (m / 8) * 128 + (r / 8) * kA2Group.
  auto resplit = [&]() {
    const int r = 32 * q + lane;
    unsigned char *rowp = A2 + (r & 7) * 16 + (r >> 3) * kA2Group;
    uint32_t v[4][XPT];
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld(tmem + lane_base + kD1 + (uint32_t)(32 * c + XPT * h), v[c]);
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld_wait_dep(v[c]);
#pragma unroll
    for (int k = 0; k < XPT / 2; ++k) {  // m = 4 XPT h + 8 k + (0..7): x = XPT h + 2 k + {0, 1}, c = 0..3
      uint4 vh, vl;
      split2<BF>(__uint_as_float(v[0][2 * k]), __uint_as_float(v[1][2 * k]), vh.x, vl.x);
      split2<BF>(__uint_as_float(v[2][2 * k]), __uint_as_float(v[3][2 * k]), vh.y, vl.y);
      split2<BF>(__uint_as_float(v[0][2 * k + 1]), __uint_as_float(v[1][2 * k + 1]), vh.z, vl.z);
      split2<BF>(__uint_as_float(v[2][2 * k + 1]), __uint_as_float(v[3][2 * k + 1]), vh.w, vl.w);
      const int mg = (XPT / 2) * h + k;
      *reinterpret_cast<uint4 *>(rowp + mg * 128) = vh;
      if (kParts == 2) *reinterpret_cast<uint4 *>(rowp + kA2Part + mg * 128) = vl;
    }
    fence_proxy_async_smem();
  };

  // ---- column MMAs: lane 0 of warp w issues output blocks j = w, w + 4, ...
  auto issue_col = [&]() {
    fence_after_sync();
#pragma unroll 1
    for (int j = warp; j < kColBlocks; j += kColIssuers) {
      const bool last = j == kColBlocks - 1;
      // K chunks of block j (the strip's kcc bounds them all)
      const int kj = kStrip && kColBlocks > 1 ? col_chunks(W, j * NBC, last ? kLastN : NBC) : kcc;
      const uint32_t idesc = last ? idesc_col_last : idesc_col;
#pragma unroll 1
      for (int i = 0; i < kj; ++i)
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
          const int ap = pp == 1 ? 1 : 0;
          const int bp = pp == 2 ? 1 : 0;
          const uint64_t bd =
              bc_desc + (uint64_t)((kStrip ? bp * kBcPart + 2 * (kcc - 1 - i) * 256 : (2 * i + bp) * NBC * 32) >> 4);
          const uint32_t ao = (uint32_t)(ap * kA2Part + (j * NBC / 16 + i) * 2 * kA2Group);
          mma_ss(tmem + kD2 + (uint32_t)(j * NBC), a2_desc + (uint64_t)(ao >> 4), bd, idesc,
                 (i > 0 || pp > 0) ? 1u : 0u);
        }
    }
    mma_commit(mbarC);
  };

  // ---- demodulate harmonic n: lane m = 32 q + lane = 4 x + c, rows y in
  // [h * BYH, (h+1) * BYH); the four lanes of one x read the same table entry.
  auto demod = [&](int n) {
    const int c = lane & 3;
    const float dn = a.d[n];
    const char *Lf =
        reinterpret_cast<const char *>(lutf + ((lbase + n) % 3) * kLutStride + ((lane >> 2) & (kCopies - 1)));
    constexpr int DG = BYH % 16 == 0 ? 16 : (BYH % 8 == 0 ? 8 : 4);  // columns per TMEM load
    uint32_t v[BYH / DG][DG];
#pragma unroll
    for (int g = 0; g < BYH / DG; ++g) tmem_ld(tmem + lane_base + kD2 + (uint32_t)(h * BYH + DG * g), v[g]);
    float t[BYH];
#pragma unroll
    for (int j = 0; j < BYH; ++j) {
      const float2 cs = *reinterpret_cast<const float2 *>(Lf + cen_off(j));
      t[j] = dn * ((c & 1) ? cs.y : cs.x);  // cos for G_r, F_r; sin for G_i, F_i
    }
#pragma unroll
    for (int g = 0; g < BYH / DG; ++g) tmem_ld_wait_dep(v[g]);
#pragma unroll
    for (int g = 0; g < BYH / DG; ++g)
#pragma unroll
      for (int j = 0; j < DG; ++j) part[DG * g + j] = fmaf(t[DG * g + j], __uint_as_float(v[g][j]), part[DG * g + j]);
  };

  // Bounded wait of this thread on an MMA barrier (each thread then reads only
  // its own TMEM lanes, so no CTA barrier is needed here); a wait that gives
  // up is recorded and agreed on at the next phase barrier.
  bool fail = false;
  auto wait_mma = [&](uint64_t *m, uint32_t &ph) {
    if (!mbar_wait_bounded(m, ph, kMaxPolls)) fail = true;
    ph ^= 1;
    fence_after_sync();
  };
  // End of a phase: CTA barrier that also agrees on failure.
  auto phase_sync = [&]() -> bool {
    fence_before_sync();
    return __syncthreads_or(fail) == 0;
  };

  for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
    const int tile_y = tile / a.tiles_x, tile_x = tile - tile_y * a.tiles_x;
    const int ty0 = tile_y * BYv, tx0 = tile_x * kBX;

    // ---- stage this tile: 128 ext rows x KX ext columns of byte offsets v * 128.
    if (tma_tile(tile)) {
      if (!mbar_wait_bounded(mbarT, phT, kMaxPolls)) *abort_s = 1;
      phT ^= 1;
      tma_pending = false;
      if (__syncthreads_or(*abort_s)) {
        ok = false;
        break;
      }
      // Box origin: column box_x(tile), row ty0 - W.  REFLECT reads the mirrored
      // source of halo pixels outside the image; pixels that touch no output
      // inside the image become the sentinel.
      const int bx0 = box_x(tile);
      if (PIPE && ty0 - W >= 0 && ty0 - W + HY <= H && tx0 - W >= 0 && tx0 - W + HX <= Wd) {
        // interior tile: every halo pixel is in the image, row ey of the box
        // (pipelined schedule only: in the serial one the extra path cost spills)
        for (int ey = warp; ey < kLanes; ey += NT / 32) {
          const unsigned char *brow = raw + ey * kBoxW + (tx0 - W - bx0);
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const int ex = lane + 32 * k4;
            if (ex < KX)
              tileT[ey * kTY + ex * kTX] = ey < HY && ex < HX ? (unsigned short)(brow[ex] * kScale) : kSent;
          }
        }
      } else {
      for (int ey = warp; ey < kLanes; ey += NT / 32) {
        const int iy = ty0 - W + ey;
        const bool row_ok = ey < HY && (reflect ? iy < H + W : (iy >= 0 && iy < H));
        const unsigned char *brow = raw + (reflect ? mirror(iy, H) - (ty0 - W) : ey) * kBoxW;
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const int ex = lane + 32 * k4;
          if (ex < KX) {
            const int ix = tx0 - W + ex;
            const bool in = row_ok && ex < HX && (reflect ? ix < Wd + W : (ix >= 0 && ix < Wd));
            const int sx = (reflect ? mirror(ix, Wd) : ix) - bx0;
            tileT[ey * kTY + ex * kTX] = in ? (unsigned short)(brow[sx] * kScale) : kSent;
          }
        }
      }
      }
      fence_proxy_async_smem();  // the box is rewritten by the next TMA copy
    } else {
      stage_tile<NT>(static_cast<const unsigned char *>(a.in), a.in_pitch, H, Wd, a.border, ty0 - W, tx0 - W, HY,
                     HX, kLanes, KX, tileT, kTX, kTY, kScale, kSent);
    }
    if (!t0_ready) build_lut<BF, NT, kParts == 1>(lut16, lutf + lbase * kLutStride, trig, 0, a.twoT, a.T, c0, tid);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    // prefetch the next tile of this CTA while this one is computed
    const int next = tile + gridDim.x;
    const int lnext = (lbase + a.K) % 3;  // the next tile's buffer of harmonic 0
    if (next < a.ntiles && tma_tile(next)) {
      if (tid == 0) issue_tma(next);
      tma_pending = true;
    }

#pragma unroll
    for (int j = 0; j < BYH; ++j) part[j] = 0.f;
    {
      const int x = 8 * q + (lane >> 2);
      const unsigned short *cen = tileT + (W + h * BYH) * kTY + (x + W) * kTX;
#pragma unroll
      for (int j = 0; j < BYH / 2; ++j)
        cen_pk[j] = (uint32_t)(cen[2 * j * kTY] >> 1) | ((uint32_t)(cen[(2 * j + 1) * kTY] >> 1) << 16);
    }

    if (!PIPE) {
      // Serial schedule: modulate -> row MMAs (tables for n+1 built meanwhile) ->
      // re-split -> column MMAs -> demodulate.
      for (int n = 0; n < a.K && ok; ++n) {
        modulate();
        if (!(ok = phase_sync())) break;
        if (row_issuer) issue_row();
        if (n + 1 < a.K)
          build_lut<BF, NT, kParts == 1>(lut16, lutf + ((lbase + n + 1) % 3) * kLutStride, trig, n + 1, a.twoT,
                                         a.T, c0, btid);
        wait_mma(mbarR, phR);
        resplit();
        if (!(ok = phase_sync())) break;
        if (col_issuer) issue_col();
        wait_mma(mbarC, phC);
        demod(n);
        if (!(ok = phase_sync())) break;
      }
    } else {
      // Pipelined schedule: the column MMAs of harmonic n run while harmonic n+1
      // is modulated, and the row MMAs of n+1 run while the tables of n+2 are
      // built and n is demodulated; two CTA barriers per harmonic.
      modulate();
      ok = phase_sync();
      if (ok) {
        if (row_issuer) issue_row();
        // harmonic m = K is the next tile's harmonic 0 (its buffer (lbase + K) % 3)
        if (a.K > 1 || next < a.ntiles)
          build_lut<BF, NT, kParts == 1>(lut16, lutf + ((lbase + 1) % 3) * kLutStride, trig, a.K > 1 ? 1 : 0,
                                         a.twoT, a.T, c0, btid);
        wait_mma(mbarR, phR);
        resplit();
        ok = phase_sync();
      }
      for (int n = 0; n < a.K && ok; ++n) {
        if (col_issuer) issue_col();  // C(n): A2 -> D2
        if (n + 1 < a.K) modulate();  // A1 <- harmonic n+1 (R(n) has finished)
        if (!(ok = phase_sync())) break;
        if (n + 1 < a.K && row_issuer) issue_row();  // R(n+1): A1 -> D1
        // Tables of n+2 while C(n) and R(n+1) run: lut16 (last read by the
        // modulation of n+1, done) and lutf buffer (lbase + n + 2) % 3 (not read
        // by demod(n) or demod(n + 1)); n + 2 = K is the next tile's harmonic 0.
        if (n + 2 < a.K || (n + 2 == a.K && next < a.ntiles))
          build_lut<BF, NT, kParts == 1>(lut16, lutf + ((lbase + n + 2) % 3) * kLutStride, trig,
                                         n + 2 < a.K ? n + 2 : 0, a.twoT, a.T, c0, btid);
        wait_mma(mbarC, phC);
        demod(n);  // D2, table n
        if (n + 1 < a.K) {
          // C(n) has finished (observed above), so A2 may be overwritten.
          wait_mma(mbarR, phR);
          resplit();  // D1 -> A2
        }
        if (!(ok = phase_sync())) break;
      }
    }
    // ---- combine the four channel partials and write fhat = P / Q.
    if (ok) {
      // [c][y][x] with the channel planes 8 floats apart in bank position, so that
      // the four channel lanes of one x store to different banks
      constexpr int kCS = BY * kBX + 8;
      float *comb = reinterpret_cast<float *>(A2);
      const int x = 8 * q + (lane >> 2), c = lane & 3;
#pragma unroll
      for (int j = 0; j < BYH; ++j) comb[c * kCS + (h * BYH + j) * kBX + x] = part[j];
      __syncthreads();
      for (int e = tid; e < BYv * kBX; e += NT) {
        const int y = e / kBX, xx = e - y * kBX;
        const int iy = ty0 + y, ix = tx0 + xx;
        if (iy < H && ix < Wd) {
          const float Q = comb[0 * kCS + y * kBX + xx] + comb[1 * kCS + y * kBX + xx];
          const float P = comb[2 * kCS + y * kBX + xx] + comb[3 * kCS + y * kBX + xx];
          *reinterpret_cast<float *>(reinterpret_cast<char *>(a.out) + (size_t)iy * a.out_pitch +
                                     (size_t)ix * sizeof(float)) = P / Q + c0;
        }
      }
    } else if (tid == 0) {
      atomicOr(&g_fbf_tc_error, 1u);
    }
    fence_before_sync();
    __syncthreads();
    t0_ready = PIPE && next < a.ntiles;  // built as harmonic K (pipelined schedule)
    lbase = PIPE ? lnext : 0;
  }
  // A prefetched box that no tile consumed (the loop was abandoned): let the
  // copy land (bounded wait) before the CTA exits.
  if (tma_pending) mbar_wait_bounded(mbarT, phT, kMaxPolls);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

#ifndef FBF_TC_NBR
#define FBF_TC_NBR 32
#endif
#ifndef FBF_TC_BY_16
#define FBF_TC_BY_16 112  // computed rows per tile, windows up to 16 (output rows min(112, 128 - 2W))
#endif
#ifndef FBF_TC_NBC_16
#define FBF_TC_NBC_16 112  // one column block (fewer, larger MMAs ran faster than 48 + 48 + 16)
#endif
#ifndef FBF_TC_NBC_64
#define FBF_TC_NBC_64 32  // split forms, 64-row tiles (a single 64-row block spilled registers there)
#endif
#ifndef FBF_TC_NBC_64_SINGLE
#define FBF_TC_NBC_64_SINGLE 64  // single FP16 form, 64-row tiles: one column block
#endif
#ifndef FBF_TC_NT_16
#define FBF_TC_NT_16 512  // threads per CTA, windows up to 16
#endif
#ifndef FBF_TC_NT_64
#define FBF_TC_NT_64 512  // threads per CTA, 64-row tiles
#endif
#ifndef FBF_TC_WMAX_96
#define FBF_TC_WMAX_96 26  // windows 17 .. this: 96 computed rows (output rows 128 - 2W), one column block
#endif
#ifndef FBF_TC_PIPE
#define FBF_TC_PIPE 1  // W <= 16: pipelined schedule (A1, D1, D2 disjoint in TMEM)
#endif

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D u8 tensor map of the input image with a kBoxW x 128 box; false when the
// base address or pitch breaks TMA's 16-byte rules (then every tile loads directly).
bool make_box_map(const FilterArgs &a, CUtensorMap *map) {
  std::memset(map, 0, sizeof(*map));
  if ((reinterpret_cast<uintptr_t>(a.in) & 15) != 0 || (a.in_pitch & 15) != 0) return false;
  if (a.in_pitch >= (1ull << 40) || a.Wd <= 0 || a.H <= 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)a.Wd, (cuuint64_t)a.H};
  const cuuint64_t strides[1] = {(cuuint64_t)a.in_pitch};
  const cuuint32_t box[2] = {(cuuint32_t)kBoxW, (cuuint32_t)kLanes};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(a.in), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BF, int NSPLIT, int BY, int WCAP, int NBR, int NBC, int PIPE, int NT>
fbf_status launch_tc_cfg(const FilterArgs &a0, cudaStream_t s) {
  FilterArgs a = a0;
  const TcLayout Ly = tc_layout(a.W, WCAP, BY, NBR, NBC);
  a.tiles_x = (a.Wd + kBX - 1) / kBX;
  const int by = tile_rows(BY, a.W);
  const int tiles_y = (a.H + by - 1) / by;
  a.ntiles = a.tiles_x * tiles_y;
  CUtensorMap map;
  const int use_tma = make_box_map(a, &map) ? 1 : 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FBF_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = a.ntiles < sms ? a.ntiles : sms;
  auto kern = fbf_tc_u8_kernel<BF, NSPLIT, BY, WCAP, NBR, NBC, PIPE, NT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Ly.bytes) != cudaSuccess)
    return FBF_ERR_CUDA;
  kern<<<grid, NT, Ly.bytes, s>>>(a, map, use_tma);
  return cuda_status(cudaGetLastError());
}

}  // namespace

// mode 0: FP16 operands, split data, single weights (2 products per step);
// 1: BF16 operands, split data and weights (3 products); 2: FP16 operands, data
// and weights rounded once (1 product; A1 then takes half the TMEM columns, so
// the tiles of windows above 16 run the pipelined schedule too); 3: BF16
// operands rounded once (second layout only: T <= 255).
fbf_status launch_tc_u8(const FilterArgs &a, int mode, cudaStream_t s) {
  if (mode < 0 || mode > 3) return FBF_ERR_INVALID_ARGUMENT;
  // The second layout (fbf_tc2_kernel.cuh) covers T <= 255 and, per form, the
  // windows of its instantiations; this kernel runs the rest.
  const fbf_status st2 = launch_tc2_u8(a, mode, s);
  if (st2 != FBF_ERR_UNSUPPORTED || mode == 3) return st2;
  constexpr int BY16 = FBF_TC_BY_16, NBC16 = FBF_TC_NBC_16, NT16 = FBF_TC_NT_16;
  if (a.W <= 16) {
    if (mode == 1) return launch_tc_cfg<1, 3, BY16, 16, FBF_TC_NBR, NBC16, FBF_TC_PIPE, NT16>(a, s);
    if (mode == 2) return launch_tc_cfg<0, 1, BY16, 16, FBF_TC_NBR, NBC16, FBF_TC_PIPE, NT16>(a, s);
    return launch_tc_cfg<0, 2, BY16, 16, FBF_TC_NBR, NBC16, FBF_TC_PIPE, NT16>(a, s);
  }
  if (a.W <= FBF_TC_WMAX_96) {
    if (mode == 1) return launch_tc_cfg<1, 3, 96, 32, FBF_TC_NBR, 96, 0, FBF_TC_NT_64>(a, s);
    if (mode == 2) return launch_tc_cfg<0, 1, 96, 32, FBF_TC_NBR, 96, 1, FBF_TC_NT_64>(a, s);
    return launch_tc_cfg<0, 2, 96, 32, FBF_TC_NBR, 96, 0, FBF_TC_NT_64>(a, s);
  }
  if (a.W <= 32) {
    if (mode == 1) return launch_tc_cfg<1, 3, 64, 32, FBF_TC_NBR, FBF_TC_NBC_64, 0, FBF_TC_NT_64>(a, s);
    if (mode == 2) return launch_tc_cfg<0, 1, 64, 32, FBF_TC_NBR, FBF_TC_NBC_64_SINGLE, 1, FBF_TC_NT_64>(a, s);
    return launch_tc_cfg<0, 2, 64, 32, FBF_TC_NBR, FBF_TC_NBC_64, 0, FBF_TC_NT_64>(a, s);
  }
  return FBF_ERR_RANGE;
}

fbf_status launch_tc2_u8(const FilterArgs &a, int mode, cudaStream_t s) {
  if (a.twoT < 2 || a.twoT > 510) return FBF_ERR_UNSUPPORTED;
  if (mode == 2) return launch_tc2_single(a, s);
  if (mode == 3) return launch_tc2_bf16_single(a, s);
  if (mode == 0) return launch_tc2_fp16(a, s);
  return launch_tc2_bf16(a, s);
}

fbf_status tc_read_clear_error(unsigned int *code) {
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_fbf_tc_error, sizeof(v)) != cudaSuccess) return FBF_ERR_CUDA;
  if (cudaMemcpyToSymbol(g_fbf_tc_error, &zero, sizeof(zero)) != cudaSuccess) return FBF_ERR_CUDA;
  *code = v;
  return FBF_OK;
}

}  // namespace fbf
