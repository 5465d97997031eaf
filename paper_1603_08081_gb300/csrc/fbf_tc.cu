// Tensor-core form of the fused shiftable bilateral filter (Algorithm 1) for
// uint8 images: both 1-D passes of every harmonic run as banded-Toeplitz
// products on the 5th-generation tensor cores (tcgen05.mma, kind::f16, FP32
// accumulation in tensor memory).
//
// One CTA (256 threads) owns a 32-column x BY-row output tile; its BY + 2W halo
// rows fit the 128 TMEM lanes (BY = 96 for W <= 16, 64 for W <= 32).  For each
// harmonic n:
//
//   modulate  thread (lane r, half h) gathers (cos, sin, f cos, f sin)(n w f)
//             for ext row r and half of the ext columns from the per-harmonic
//             table, splits each value into hi + lo 16-bit parts and writes
//             them with tcgen05.st into TMEM: A1[c][part] (lane = ext row,
//             K = ext column, two 16-bit elements per 32-bit column);
//   row MMA   D1[c] (lane = ext row, 32 columns = outputs x) = sum over
//             16-wide K chunks of A1[c][part] * T_i[part]; T_i is the 16 x 16
//             Toeplitz block of chunk offset i (entries w[16 i + k - n]), the
//             same block for every output block (banded: only the
//             ceil((16 + 2W) / 16) chunks that meet the band are issued);
//   re-split  D1 rows are read back (tcgen05.ld), split into hi / lo again
//             and stored to shared memory as the MN-major A operand of the
//             column pass, A2[m = c * 32 + x][K = ext row] -- each thread
//             writes its own row, so no transpose is needed;
//   col MMA   D2 (lane m = (c, x), columns = output rows y) = sum A2 * T_i;
//   demod     lane (c, x) accumulates d_n * trig(n w f(y, x)) * D2 into its
//             own partial: cos for the G_r / F_r channels, sin for G_i / F_i.
//
// P = partial(F_r) + partial(F_i), Q = partial(G_r) + partial(G_i) are combined
// once per tile, and fhat = P / Q is written.  Precision: the data are split
// hi + lo; FP16 uses one weight part (2 products per step), BF16 splits the
// weights too (3 products).  Table entries, the phase (exact integer
// reduction), the K-term accumulation and the ratio stay in FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fbf_internal.h"
#include "fbf_tc_ptx.cuh"

__device__ unsigned int g_fbf_tc_error = 0;

namespace fbf {
namespace {

using namespace tc;

constexpr int kCopies = 8;
constexpr int kLutEntries = 257;
constexpr int kSentinel = 256;
constexpr int kLutStride = kLutEntries * kCopies;  // float4 per table buffer
constexpr int kBX = 32;                             // output columns per tile
constexpr int kLanes = 128;                         // TMEM lanes = halo rows per tile
constexpr int kPT = kLanes + 2;                     // tile pitch (u16), PT/2 odd
constexpr int kA2Group = 2048;                      // bytes per 8-row K group of A2 (16 M groups x 128 B)
constexpr int kA2Part = 16 * kA2Group;              // one part of A2: 128 (M) x 128 (K) x 16 bit
constexpr uint32_t kMaxPolls = 1u << 22;
constexpr int kNT = 256;

struct TcLayout {
  int kc;   // 16-wide K chunks meeting the band of one 16-output block
  int KX;   // K extent of the row pass (ext columns, multiple of 16)
  int A1C;  // TMEM columns per (channel, part) of A1 = KX / 2
  size_t lut_off, a2_off, b_off, tile_off, bar_off, bytes;
};

__host__ __device__ inline TcLayout tc_layout(int W, int wcap) {
  TcLayout L;
  L.kc = (16 + 2 * W + 15) / 16;
  L.KX = 16 * (kBX / 16 - 1 + L.kc);
  L.A1C = L.KX / 2;
  const int kcmax = (16 + 2 * wcap + 15) / 16;
  const int KXmax = 16 * (kBX / 16 - 1 + kcmax);
  L.lut_off = 0;
  L.a2_off = L.lut_off + 2ull * kLutStride * sizeof(float4);
  L.b_off = L.a2_off + 2ull * kA2Part;
  L.tile_off = L.b_off + (size_t)kcmax * 2 * 512;
  L.bar_off = L.tile_off + (((size_t)KXmax * kPT * 2 + 127) & ~(size_t)127);
  L.bytes = L.bar_off + 64;
  return L;
}

__device__ __forceinline__ int reflect_index(int i, int n) {
  const int p = 2 * n;
  int m = i % p;
  if (m < 0) m += p;
  return m < n ? m : p - 1 - m;
}

__device__ __forceinline__ void build_lut(float4 *L, int n, int twoT, float T, int tid) {
  for (int v = tid; v < 256; v += kNT) {
    const int m = (n * v) % twoT;
    float sn, cs;
    sincospif((float)m / T, &sn, &cs);
    const float fv = (float)v;
    const float4 e = make_float4(cs, sn, fv * cs, fv * sn);
#pragma unroll
    for (int j = 0; j < kCopies; ++j) L[v * kCopies + ((j + v) & (kCopies - 1))] = e;
  }
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

__device__ __forceinline__ void tmem_st_x4(uint32_t taddr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r0), "r"(r1),
               "r"(r2), "r"(r3)
               : "memory");
}

// BF: 0 = FP16, 1 = BF16.  NSPLIT: 2 = data hi/lo x weights hi; 3 = plus data hi x weights lo.
// BY: output rows per tile (BY + 2 * WCAP <= 128).
template <int BF, int NSPLIT, int BY, int WCAP>
__global__ void __launch_bounds__(kNT, 1) fbf_tc_u8_kernel(const __grid_constant__ FilterArgs a) {
  static_assert(BY + 2 * WCAP <= kLanes && BY % 32 == 0, "halo rows must fit the TMEM lanes");
  constexpr int BYH = BY / 2;  // output rows per thread in the demodulation
  extern __shared__ __align__(1024) unsigned char smem[];
  const int W = a.W;
  const TcLayout Ly = tc_layout(W, WCAP);
  float4 *lut = reinterpret_cast<float4 *>(smem + Ly.lut_off);
  unsigned char *A2 = smem + Ly.a2_off;
  unsigned char *Bt = smem + Ly.b_off;
  unsigned short *tileT = reinterpret_cast<unsigned short *>(smem + Ly.tile_off);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Ly.bar_off);
  uint32_t *tmem_base_s = reinterpret_cast<uint32_t *>(smem + Ly.bar_off + 16);
  int *abort_s = reinterpret_cast<int *>(smem + Ly.bar_off + 32);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quadrant, half
  const int tile_y = blockIdx.x / a.tiles_x, tile_x = blockIdx.x - tile_y * a.tiles_x;
  const int ty0 = tile_y * BY, tx0 = tile_x * kBX;
  const int H = a.H, Wd = a.Wd, HY = BY + 2 * W;
  const int kc = Ly.kc, A1C = Ly.A1C;

  if (warp == 0) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(mbar, 1);
    mbar_fence_init();
    *abort_s = 0;
  }
  if (tid < 2 * kCopies)
    lut[(tid / kCopies) * kLutStride + kSentinel * kCopies + (tid % kCopies)] = make_float4(0.f, 0.f, 0.f, 0.f);

  // Toeplitz blocks T_i (16 x 16, K-major, no swizzle): element (n, k) = w[16 i + k - n]
  // inside the band, 0 outside; part 0 = hi, part 1 = lo residual of the weights.
  for (int e = tid; e < kc * 256; e += kNT) {
    const int i = e >> 8, n = (e >> 4) & 15, k = e & 15;
    const int t = 16 * i + k - n;
    const float wv = (t >= 0 && t <= 2 * W) ? a.w[t] : 0.f;
    const unsigned short hi = to16<BF>(wv);
    const unsigned short lo = to16<BF>(wv - from16<BF>(hi));
    const int off = (n & 7) * 16 + (n >> 3) * 256 + (k & 7) * 2 + (k >> 3) * 128;
    *reinterpret_cast<unsigned short *>(Bt + (size_t)i * 1024 + off) = hi;
    *reinterpret_cast<unsigned short *>(Bt + (size_t)i * 1024 + 512 + off) = lo;
  }

  // Halo tile, transposed, as byte offsets into a table buffer (sentinel outside).
  {
    const unsigned char *in = static_cast<const unsigned char *>(a.in);
    const size_t pitch = a.in_pitch;
    const int KX = Ly.KX, total = kLanes * KX;
    const int HX = kBX + 2 * W;
    for (int base = tid; base < total; base += kNT * 8) {
      unsigned short vals[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * kNT;
        unsigned short v = kSentinel * kCopies * sizeof(float4);
        if (idx < total) {
          const int ey = idx / KX, ex = idx - ey * KX;
          if (ey < HY && ex < HX) {
            int iy = ty0 + ey - W, ix = tx0 + ex - W;
            bool inside;
            if (a.border == FBF_BORDER_REFLECT) {
              iy = reflect_index(iy, H);
              ix = reflect_index(ix, Wd);
              inside = true;
            } else {
              inside = iy >= 0 && iy < H && ix >= 0 && ix < Wd;
            }
            if (inside) v = (unsigned short)(__ldg(in + (size_t)iy * pitch + ix) * (kCopies * sizeof(float4)));
          }
        }
        vals[u] = v;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * kNT;
        if (idx < total) {
          const int ey = idx / KX, ex = idx - ey * KX;
          tileT[ex * kPT + ey] = vals[u];
        }
      }
    }
  }
  build_lut(lut, 0, a.twoT, a.T, tid);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_base_s;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  const uint32_t kA1 = 0, kD1 = 384, kD2 = 0;  // TMEM column bases (D2 reuses A1's columns)
  constexpr uint32_t idesc_row = idesc_f16(128, 16, BF, 0, 0);
  constexpr uint32_t idesc_col = idesc_f16(128, 16, BF, 1, 0);
  const uint32_t b_s = smem_u32(Bt), a2_s = smem_u32(A2);

  float part[BYH];
#pragma unroll
  for (int j = 0; j < BYH; ++j) part[j] = 0.f;
  uint32_t phase = 0;
  bool ok = true;

  for (int n = 0; n < a.K && ok; ++n) {
    const char *Lc = reinterpret_cast<const char *>(lut + (n & 1) * kLutStride + (lane & (kCopies - 1)));

    // ---- modulate: ext row r = 32 q + lane, columns [h * A1C/2, (h+1) * A1C/2) in pairs.
    {
      const int r = 32 * q + lane;
      const int c0 = h * (A1C / 2), c1 = (h + 1) * (A1C / 2);
      for (int col = c0; col < c1; col += 4) {
        uint32_t hi[4][4], lo[4][4];  // [channel][column]
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int u = 2 * (col + j);
          const float4 e0 = *reinterpret_cast<const float4 *>(Lc + tileT[u * kPT + r]);
          const float4 e1 = *reinterpret_cast<const float4 *>(Lc + tileT[(u + 1) * kPT + r]);
          split2<BF>(e0.x, e1.x, hi[0][j], lo[0][j]);
          split2<BF>(e0.y, e1.y, hi[1][j], lo[1][j]);
          split2<BF>(e0.z, e1.z, hi[2][j], lo[2][j]);
          split2<BF>(e0.w, e1.w, hi[3][j], lo[3][j]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t t_hi = tmem + lane_base + kA1 + (uint32_t)((2 * c) * A1C + col);
          const uint32_t t_lo = tmem + lane_base + kA1 + (uint32_t)((2 * c + 1) * A1C + col);
          tmem_st_x4(t_hi, hi[c][0], hi[c][1], hi[c][2], hi[c][3]);
          tmem_st_x4(t_lo, lo[c][0], lo[c][1], lo[c][2], lo[c][3]);
        }
      }
      tmem_st_wait();
    }
    fence_before_sync();
    __syncthreads();

    // ---- row MMAs (one thread), then build the next table while they run.
    if (tid == 0) {
      fence_after_sync();
#pragma unroll 1
      for (int c = 0; c < 4; ++c)
#pragma unroll 1
        for (int j = 0; j < kBX / 16; ++j)
#pragma unroll 1
          for (int i = 0; i < kc; ++i) {
            const uint32_t d = tmem + kD1 + (uint32_t)(c * 32 + j * 16);
            const uint32_t ahi = tmem + kA1 + (uint32_t)((2 * c) * A1C + (j + i) * 8);
            const uint32_t alo = tmem + kA1 + (uint32_t)((2 * c + 1) * A1C + (j + i) * 8);
            const uint64_t bhi = smem_desc(b_s + i * 1024, 128, 256);
            mma_ts(d, ahi, bhi, idesc_row, i > 0 ? 1u : 0u);
            mma_ts(d, alo, bhi, idesc_row, 1u);
            if (NSPLIT == 3) mma_ts(d, ahi, smem_desc(b_s + i * 1024 + 512, 128, 256), idesc_row, 1u);
          }
      mma_commit(mbar);
    }
    if (n + 1 < a.K) build_lut(lut + ((n + 1) & 1) * kLutStride, n + 1, a.twoT, a.T, tid);
    if (!mbar_wait_bounded(mbar, phase, kMaxPolls)) *abort_s = 1;
    phase ^= 1;
    fence_after_sync();
    if (__syncthreads_or(*abort_s)) {
      ok = false;
      break;
    }

    // ---- re-split the row-pass result into the column pass's A operand.
    // Thread: ext row r, channels 2h and 2h+1; A2[m = c*32 + x][r] is MN-major:
    // (m % 8) * 2 + (r % 8) * 16 + (m / 8) * 128 + (r / 8) * kA2Group.
    {
      const int r = 32 * q + lane;
      unsigned char *rowp = A2 + (r & 7) * 16 + (r >> 3) * kA2Group;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int c = 2 * h + cc;
#pragma unroll
        for (int half16 = 0; half16 < 2; ++half16) {
          uint32_t v[16];
          tmem_ld_x16(tmem + lane_base + kD1 + (uint32_t)(c * 32 + half16 * 16), v);
          tmem_ld_wait();
#pragma unroll
          for (int g = 0; g < 2; ++g) {  // 8 consecutive m = one 16-byte row of a core matrix
            uint4 vh, vl;
            split2<BF>(__uint_as_float(v[8 * g + 0]), __uint_as_float(v[8 * g + 1]), vh.x, vl.x);
            split2<BF>(__uint_as_float(v[8 * g + 2]), __uint_as_float(v[8 * g + 3]), vh.y, vl.y);
            split2<BF>(__uint_as_float(v[8 * g + 4]), __uint_as_float(v[8 * g + 5]), vh.z, vl.z);
            split2<BF>(__uint_as_float(v[8 * g + 6]), __uint_as_float(v[8 * g + 7]), vh.w, vl.w);
            const int mg = c * 4 + half16 * 2 + g;  // M group of 8
            *reinterpret_cast<uint4 *>(rowp + mg * 128) = vh;
            *reinterpret_cast<uint4 *>(rowp + kA2Part + mg * 128) = vl;
          }
        }
      }
    }
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();

    // ---- column MMAs.
    if (tid == 0) {
      fence_after_sync();
#pragma unroll 1
      for (int j = 0; j < BY / 16; ++j)
#pragma unroll 1
        for (int i = 0; i < kc; ++i) {
          const uint32_t d = tmem + kD2 + (uint32_t)(j * 16);
          const uint32_t ao = (uint32_t)((j + i) * 2 * kA2Group);
          const uint64_t ahi = smem_desc(a2_s + ao, kA2Group, 128);
          const uint64_t alo = smem_desc(a2_s + kA2Part + ao, kA2Group, 128);
          const uint64_t bhi = smem_desc(b_s + i * 1024, 128, 256);
          mma_ss(d, ahi, bhi, idesc_col, i > 0 ? 1u : 0u);
          mma_ss(d, alo, bhi, idesc_col, 1u);
          if (NSPLIT == 3) mma_ss(d, ahi, smem_desc(b_s + i * 1024 + 512, 128, 256), idesc_col, 1u);
        }
      mma_commit(mbar);
    }
    if (!mbar_wait_bounded(mbar, phase, kMaxPolls)) *abort_s = 1;
    phase ^= 1;
    fence_after_sync();
    if (__syncthreads_or(*abort_s)) {
      ok = false;
      break;
    }

    // ---- demodulate: lane m = c * 32 + x (c = q), rows y in [h * BYH, (h+1) * BYH).
    {
      const int x = lane;
      const float dn = a.d[n];
      const int trig = q & 1;  // 0: cos (G_r, F_r), 1: sin (G_i, F_i)
      const unsigned short *cen = tileT + (x + W) * kPT + W + h * BYH;
#pragma unroll
      for (int y0 = 0; y0 < BYH; y0 += 16) {
        uint32_t v[16];
        tmem_ld_x16(tmem + lane_base + kD2 + (uint32_t)(h * BYH + y0), v);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 cs = *reinterpret_cast<const float2 *>(Lc + cen[y0 + j]);
          const float t = trig ? cs.y : cs.x;
          part[y0 + j] = fmaf(dn * t, __uint_as_float(v[j]), part[y0 + j]);
        }
      }
    }
    fence_before_sync();
    __syncthreads();
  }

  // ---- combine the four channel partials and write fhat = P / Q.
  if (ok) {
    float *comb = reinterpret_cast<float *>(A2);  // [c][y][x], 4 * BY * 32 floats
#pragma unroll
    for (int j = 0; j < BYH; ++j) comb[(q * BY + h * BYH + j) * kBX + lane] = part[j];
    __syncthreads();
    for (int e = tid; e < BY * kBX; e += kNT) {
      const int y = e / kBX, x = e - y * kBX;
      const int iy = ty0 + y, ix = tx0 + x;
      if (iy < H && ix < Wd) {
        const float Q = comb[(0 * BY + y) * kBX + x] + comb[(1 * BY + y) * kBX + x];
        const float P = comb[(2 * BY + y) * kBX + x] + comb[(3 * BY + y) * kBX + x];
        *reinterpret_cast<float *>(reinterpret_cast<char *>(a.out) + (size_t)iy * a.out_pitch +
                                   (size_t)ix * sizeof(float)) = P / Q;
      }
    }
  } else if (tid == 0) {
    atomicOr(&g_fbf_tc_error, 1u);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

template <int BF, int NSPLIT, int BY, int WCAP>
fbf_status launch_tc_cfg(const FilterArgs &a0, cudaStream_t s) {
  FilterArgs a = a0;
  const TcLayout Ly = tc_layout(a.W, WCAP);
  a.tiles_x = (a.Wd + kBX - 1) / kBX;
  const int tiles_y = (a.H + BY - 1) / BY;
  a.ntiles = a.tiles_x * tiles_y;
  auto kern = fbf_tc_u8_kernel<BF, NSPLIT, BY, WCAP>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Ly.bytes) != cudaSuccess)
    return FBF_ERR_CUDA;
  kern<<<a.ntiles, kNT, Ly.bytes, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace

// bf16 != 0: BF16 operands with split weights (3 products per step);
// otherwise FP16 operands, split data, single weights (2 products).
fbf_status launch_tc_u8(const FilterArgs &a, int bf16, cudaStream_t s) {
  if (a.W <= 16) return bf16 ? launch_tc_cfg<1, 3, 96, 16>(a, s) : launch_tc_cfg<0, 2, 96, 16>(a, s);
  if (a.W <= 32) return bf16 ? launch_tc_cfg<1, 3, 64, 32>(a, s) : launch_tc_cfg<0, 2, 64, 32>(a, s);
  return FBF_ERR_RANGE;
}

fbf_status tc_read_clear_error(unsigned int *code) {
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_fbf_tc_error, sizeof(v)) != cudaSuccess) return FBF_ERR_CUDA;
  if (cudaMemcpyToSymbol(g_fbf_tc_error, &zero, sizeof(zero)) != cudaSuccess) return FBF_ERR_CUDA;
  *code = v;
  return FBF_OK;
}

}  // namespace fbf
