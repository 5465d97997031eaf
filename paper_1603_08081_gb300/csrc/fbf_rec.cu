// Algorithm 1 with the recursive Gaussian (the constant-time Gaussian filtering
// that Sec. II cites after eq. (5): Deriche's fourth-order approximation) for
// uint8 images, FP32.  The cost per pixel and harmonic does not depend on
// sigma_s: each 1-D pass is a causal and an anticausal recursion of two
// second-order sections per channel (coefficients from recursive_coeffs).
//
// Per chunk of harmonics (all of them when the scratch fits 4 GiB), three
// kernels, one thread per image line, harmonic and channel pair (cos, sin) or
// ((f - T/2) cos, (f - T/2) sin):
//   rec_v    thread (column x, harmonic n): modulates f(y, x) on the fly into
//            the four real channels (cos, sin, (f - T/2) cos, (f - T/2) sin)(n w f)
//            (exact integer phase n f mod 2T, a 256-entry table per block), runs
//            the causal recursion down the column and the anticausal one up
//            it, and writes their sum to vt[n][c][x][y] -- transposed, through a
//            32 x 32 shared-memory tile per channel (the causal half waits in
//            the s2 planes in natural layout), so that every global access of
//            both passes is coalesced;
//   rec_h    thread (row y, harmonic n): the same recursions along x on vt
//            (consecutive threads read consecutive y: coalesced), the causal
//            result kept in s2 (same layout), then demodulation:
//            P_n = d_n (cos, sin) . (Fr, Fi) or Q_n = d_n (cos, sin) . (Gr, Gi);
//   rec_out  sums (P_n, Q_n) over the chunk (and the chunks before it) and, on
//            the last chunk, writes fhat = P / Q + T/2 through a tile transpose.
// Borders: TRUNCATE is zero outside the image; REFLECT extends every line by E
// mirrored samples on each side (half-sample symmetric, repeated), zero beyond.
// Scratch: 40 bytes per pixel and harmonic of the chunk, plus 8 per pixel,
// allocated and freed stream-ordered from the library's pool.
#include <cuda_runtime.h>

#include <algorithm>

#include "fbf_common.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kChunk = 16;  // vertical pass: steps whose loads are issued together
constexpr int kChunkA = 8;  // its anticausal half (four more loads per step)
constexpr int kChunkH = 8;  // horizontal pass: the same

struct RecArgs {
  const unsigned char *in;
  size_t in_pitch;
  float *out;
  size_t out_pitch;
  int H, Wd, twoT, border, E;
  int n0, nh, first, last;  // harmonics n0 .. n0 + nh - 1; first / last chunk
  float T, c0;
  float rn[2][2], rm[2][2], rp[2][2];
  float *vt;    // [nh][4][Wd][H] vertical pass, transposed
  float *s2;    // [nh][4] planes: causal half of the vertical pass ([y][x]), then of the horizontal one ([x][y])
  float *pq;    // [nh][2][Wd][H] P_n and Q_n planes
  float2 *acc;  // [Wd][H]        (P, Q) of the chunks so far
  float d[FBF_KMAX];
};

// (cos, sin)(pi m / T), m = n v mod 2T, for v = 0..255 (exact integer phase),
// times (v - T/2) when `weighted` (the channels of the f-weighted pair).
__device__ __forceinline__ void build_tab(float2 *tab, int n, const RecArgs &r, bool weighted) {
  for (int v = threadIdx.x + threadIdx.y * blockDim.x; v < 256; v += blockDim.x * blockDim.y) {
    const int m = (int)(((long long)n * v) % r.twoT);
    float sn, cs;
    sincospif((float)m / r.T, &sn, &cs);
    const float fv = weighted ? (float)v - r.c0 : 1.f;
    tab[v] = make_float2(fv * cs, fv * sn);
  }
  __syncthreads();
}

// One step of the causal recursion (both sections, the thread's two channels): input c,
// state x1 (previous input), y1, y2 (previous outputs per section); returns
// the sum of the sections in yo.
struct Causal {
  float x1[2] = {}, y1[2][2] = {}, y2[2][2] = {};
  __device__ __forceinline__ void step(const RecArgs &r, const float (&c)[2], float (&yo)[2]) {
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float yn = fmaf(-r.rp[i][0], y1[i][ch],
                              fmaf(r.rn[i][0], c[ch], fmaf(r.rn[i][1], x1[ch], -r.rp[i][1] * y2[i][ch])));
        y2[i][ch] = y1[i][ch];
        y1[i][ch] = yn;
      }
      yo[ch] = y1[0][ch] + y1[1][ch];
      x1[ch] = c[ch];
    }
  }
};
// The anticausal recursion, run backwards: the output at k uses the inputs at
// k + 1, k + 2 (x1, x2) and the outputs at k + 1, k + 2; then takes input c.
struct Anticausal {
  float x1[2] = {}, x2[2] = {}, z1[2][2] = {}, z2[2][2] = {};
  __device__ __forceinline__ void step(const RecArgs &r, const float (&c)[2], float (&yo)[2]) {
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float zn = fmaf(-r.rp[i][0], z1[i][ch],
                              fmaf(r.rm[i][0], x1[ch], fmaf(r.rm[i][1], x2[ch], -r.rp[i][1] * z2[i][ch])));
        z2[i][ch] = z1[i][ch];
        z1[i][ch] = zn;
      }
      yo[ch] = z1[0][ch] + z1[1][ch];
      x2[ch] = x1[ch];
      x1[ch] = c[ch];
    }
  }
};

__global__ void __launch_bounds__(32) fbf_rec_v_kernel(const __grid_constant__ RecArgs r) {
  __shared__ float2 tab[256];
  __shared__ float tile[2][32][33];  // [channel of the pair][column in block][row in group]
  // channel pair cp = blockIdx.z: 0 = (cos, sin), 1 = ((f - T/2) cos, (f - T/2) sin)
  const int lane = threadIdx.x, x0 = blockIdx.x * 32, x = x0 + lane, nl = blockIdx.y, cp = blockIdx.z;
  build_tab(tab, r.n0 + nl, r, cp != 0);  // tab[v]: the pair's two channels of pixel value v
  const int H = r.H, Wd = r.Wd;
  const bool reflect = r.border == FBF_BORDER_REFLECT;
  const int E = reflect ? r.E : 0;
  const int xs = x < Wd ? x : Wd - 1;  // lanes past the image compute on a clamped column, store nothing
  const size_t plane = (size_t)Wd * H, ip = r.in_pitch;
  float *vt = r.vt + ((size_t)nl * 4 + 2 * cp) * plane;
  const unsigned char *col = r.in + xs;  // this thread's column
  // pixel of extended row ye, or -1 outside a TRUNCATE image
  auto load = [&](int ye) -> int {
    if (!reflect && (ye < 0 || ye >= H)) return -1;
    const int sy = reflect ? reflect_index(ye, H) : ye;
    return __ldg(col + (size_t)sy * ip);
  };
  auto chan = [&](int v, float (&c)[2]) {
    const float2 t = v < 0 ? make_float2(0.f, 0.f) : tab[v];
    c[0] = t.x;
    c[1] = t.y;
  };
  // the tile of rows [base, last] to vt: lane = row offset (coalesced); a full
  // tile (32 columns inside the image, 32 rows) without per-store checks
  const bool full_cols = x0 + 32 <= Wd;
  auto flush = [&](int base, int lastrow) {
    __syncwarp();
    const int y = base + lane;
    if (full_cols && lastrow == base + 31) {
      float *q = vt + (size_t)x0 * H + y;
#pragma unroll 8
      for (int xl = 0; xl < 32; ++xl, q += H) {
        q[0] = tile[0][xl][lane];
        q[plane] = tile[1][xl][lane];
      }
    } else {
      for (int ch = 0; ch < 2; ++ch)
        for (int xl = 0; xl < 32 && x0 + xl < Wd; ++xl)
          if (y <= lastrow) vt[((size_t)ch * Wd + x0 + xl) * H + y] = tile[ch][xl][lane];
    }
    __syncwarp();
  };
  // The loads of a chunk of steps are issued together, then the recursion runs
  // over them: one load latency per chunk instead of one per step.  The causal
  // half goes to s2 in natural layout ([c][y][x], coalesced over the lanes);
  // the anticausal pass reads it back with its own loads and writes the sum
  // to vt through the transposing tile.  Chunks wholly inside the image take
  // strided pointers and no border logic.
  float *sh = r.s2 + ((size_t)nl * 4 + 2 * cp) * plane;
  const bool xin = x < Wd;
  Causal cz;
  for (int y0 = -E; y0 < H + E; y0 += kChunk) {
    int vv[kChunk];
    if (y0 >= 0 && y0 + kChunk <= H) {
      const unsigned char *p = col + (size_t)y0 * ip;
#pragma unroll
      for (int j = 0; j < kChunk; ++j) vv[j] = __ldg(p + j * ip);
      float *q = sh + (size_t)y0 * Wd + xs;
#pragma unroll
      for (int j = 0; j < kChunk; ++j, q += Wd) {
        float c[2], yo[2];
        chan(vv[j], c);
        cz.step(r, c, yo);
        if (xin) {
          q[0] = yo[0];
          q[plane] = yo[1];
        }
      }
      continue;
    }
    const int y1 = y0 + kChunk - 1;
    if (reflect && y1 < H + E && ((y0 >= -H && y1 < 0) || (y0 >= H && y1 < 2 * H))) {
      // extension rows mirrored once: source rows s0, s0 - 1, ... (no output)
      const int s0 = y1 < 0 ? -1 - y0 : 2 * H - 1 - y0;
      const unsigned char *p = col + (size_t)s0 * ip;
#pragma unroll
      for (int j = 0; j < kChunk; ++j) vv[j] = __ldg(p - (size_t)j * ip);
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        float c[2], yo[2];
        chan(vv[j], c);
        cz.step(r, c, yo);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < kChunk; ++j) vv[j] = y0 + j < H + E ? load(y0 + j) : -1;
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const int ye = y0 + j;
      if (ye >= H + E) break;
      float c[2], yo[2];
      chan(vv[j], c);
      cz.step(r, c, yo);
      if (xin && ye >= 0 && ye < H) {
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) sh[(size_t)ch * plane + (size_t)ye * Wd + x] = yo[ch];
      }
    }
  }
  Anticausal az;
  for (int y0 = H + E - 1; y0 >= -E; y0 -= kChunkA) {
    int vv[kChunkA];
    float sv[kChunkA][2];
    if (y0 - (kChunkA - 1) >= 0 && y0 < H) {
      const unsigned char *p = col + (size_t)y0 * ip;
      const float *q = sh + (size_t)y0 * Wd + xs;  // clamped column: in bounds, unused past the image
#pragma unroll
      for (int j = 0; j < kChunkA; ++j) {
        vv[j] = __ldg(p - (size_t)j * ip);
        sv[j][0] = q[-(ptrdiff_t)j * Wd];
        sv[j][1] = q[plane - (size_t)j * Wd];
      }
#pragma unroll
      for (int j = 0; j < kChunkA; ++j) {
        const int ye = y0 - j;
        float c[2], yo[2];
        chan(vv[j], c);
        az.step(r, c, yo);
        tile[0][lane][ye & 31] = yo[0] + sv[j][0];
        tile[1][lane][ye & 31] = yo[1] + sv[j][1];
        if ((ye & 31) == 0) flush(ye, ye + 31 < H - 1 ? ye + 31 : H - 1);
      }
      continue;
    }
    const int y1 = y0 - (kChunkA - 1);
    if (reflect && y1 >= -E && ((y1 >= H && y0 < 2 * H) || (y1 >= -H && y0 < 0))) {
      // extension rows mirrored once: source rows s0, s0 + 1, ... (no output)
      const int s0 = y0 < 0 ? -1 - y0 : 2 * H - 1 - y0;
      const unsigned char *p = col + (size_t)s0 * ip;
#pragma unroll
      for (int j = 0; j < kChunkA; ++j) vv[j] = __ldg(p + (size_t)j * ip);
#pragma unroll
      for (int j = 0; j < kChunkA; ++j) {
        float c[2], yo[2];
        chan(vv[j], c);
        az.step(r, c, yo);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < kChunkA; ++j) {
      const int ye = y0 - j;
      vv[j] = ye >= -E ? load(ye) : -1;
      const bool out = xin && ye >= 0 && ye < H;
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) sv[j][ch] = out ? sh[(size_t)ch * plane + (size_t)ye * Wd + x] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < kChunkA; ++j) {
      const int ye = y0 - j;
      if (ye < -E) break;
      float c[2], yo[2];
      chan(vv[j], c);
      az.step(r, c, yo);
      if (ye >= 0 && ye < H) {
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) tile[ch][lane][ye & 31] = yo[ch] + sv[j][ch];
        if ((ye & 31) == 0) flush(ye, ye + 31 < H - 1 ? ye + 31 : H - 1);
      }
    }
  }
}

__global__ void __launch_bounds__(32) fbf_rec_h_kernel(const __grid_constant__ RecArgs r) {
  __shared__ float2 tab[256];
  const int lane = threadIdx.x, y = blockIdx.x * 32 + lane, nl = blockIdx.y, n = r.n0 + nl, cp = blockIdx.z;
  build_tab(tab, n, r, false);  // the plain (cos, sin) for the demodulation
  const int H = r.H, Wd = r.Wd;
  const bool reflect = r.border == FBF_BORDER_REFLECT;
  const int E = reflect ? r.E : 0;
  const bool yin = y < H;
  const int yc = yin ? y : H - 1;  // rows past the image load from a clamped row, store nothing
  const size_t plane = (size_t)Wd * H;
  const float *vt = r.vt + ((size_t)nl * 4 + 2 * cp) * plane;
  float *s2 = r.s2 + ((size_t)nl * 4 + 2 * cp) * plane;
  float *pq = r.pq + ((size_t)nl * 2 + (cp ? 0 : 1)) * plane;  // P plane (cp 1) or Q plane (cp 0)
  const float dn = r.d[n];
  auto chan = [&](int xe, float (&c)[2]) {
    const bool in_img = xe >= 0 && xe < Wd;
    if (!yin || (!reflect && !in_img) || xe < -E || xe >= Wd + E) {
      c[0] = c[1] = 0.f;
      return;
    }
    const int sx = reflect ? reflect_index(xe, Wd) : xe;
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) c[ch] = vt[(size_t)ch * plane + (size_t)sx * H + y];
  };
  // kChunkH steps' loads are issued together (see rec_v); chunks wholly inside
  // the image take strided pointers and no border logic
  Causal cz;
  for (int x0 = -E; x0 < Wd + E; x0 += kChunkH) {
    float cc[kChunkH][2];
    if (x0 >= 0 && x0 + kChunkH <= Wd) {
      const float *p = vt + (size_t)x0 * H + yc;
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        cc[j][0] = p[(size_t)j * H];
        cc[j][1] = p[plane + (size_t)j * H];
      }
      float *q = s2 + (size_t)x0 * H + yc;
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        float yo[2];
        cz.step(r, cc[j], yo);
        if (yin) {
          q[(size_t)j * H] = yo[0];
          q[plane + (size_t)j * H] = yo[1];
        }
      }
      continue;
    }
    const int x1 = x0 + kChunkH - 1;
    if (reflect && x1 < Wd + E && ((x0 >= -Wd && x1 < 0) || (x0 >= Wd && x1 < 2 * Wd))) {
      // extension columns mirrored once: source columns s0, s0 - 1, ... (no output)
      const int s0 = x1 < 0 ? -1 - x0 : 2 * Wd - 1 - x0;
      const float *p = vt + (size_t)s0 * H + yc;
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        cc[j][0] = p[-(ptrdiff_t)j * H];
        cc[j][1] = p[plane - (size_t)j * H];
      }
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        float yo[2];
        cz.step(r, cc[j], yo);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < kChunkH; ++j) chan(x0 + j, cc[j]);
#pragma unroll
    for (int j = 0; j < kChunkH; ++j) {
      const int xe = x0 + j;
      if (xe >= Wd + E) break;
      float yo[2];
      cz.step(r, cc[j], yo);
      if (yin && xe >= 0 && xe < Wd) {
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) s2[(size_t)ch * plane + (size_t)xe * H + y] = yo[ch];
      }
    }
  }
  Anticausal az;
  const unsigned char *row = r.in + (size_t)(yin ? y : 0) * r.in_pitch;
  const unsigned char *rowc = r.in + (size_t)yc * r.in_pitch;
  for (int x0 = Wd + E - 1; x0 >= -E; x0 -= kChunkH) {
    float cc[kChunkH][2], sv[kChunkH][2];
    int fv[kChunkH];
    if (x0 - (kChunkH - 1) >= 0 && x0 < Wd) {
      const float *p = vt + (size_t)x0 * H + yc;
      const float *q = s2 + (size_t)x0 * H + yc;
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        cc[j][0] = p[-(ptrdiff_t)j * H];
        cc[j][1] = p[plane - (size_t)j * H];
        sv[j][0] = q[-(ptrdiff_t)j * H];
        sv[j][1] = q[plane - (size_t)j * H];
        fv[j] = __ldg(rowc + x0 - j);
      }
      float *o = pq + (size_t)x0 * H + yc;
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        float yo[2];
        az.step(r, cc[j], yo);
        if (yin) {
          const float2 cs = tab[fv[j]];
          o[-(ptrdiff_t)j * H] = dn * fmaf(cs.x, yo[0] + sv[j][0], cs.y * (yo[1] + sv[j][1]));
        }
      }
      continue;
    }
    const int x1 = x0 - (kChunkH - 1);
    if (reflect && x1 >= -E && ((x1 >= Wd && x0 < 2 * Wd) || (x1 >= -Wd && x0 < 0))) {
      // extension columns mirrored once: source columns s0, s0 + 1, ... (no output)
      const int s0 = x0 < 0 ? -1 - x0 : 2 * Wd - 1 - x0;
      const float *p = vt + (size_t)s0 * H + yc;
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        cc[j][0] = p[(size_t)j * H];
        cc[j][1] = p[plane + (size_t)j * H];
      }
#pragma unroll
      for (int j = 0; j < kChunkH; ++j) {
        float yo[2];
        az.step(r, cc[j], yo);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < kChunkH; ++j) {
      const int xe = x0 - j;
      chan(xe, cc[j]);
      const bool out = yin && xe >= 0 && xe < Wd;
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) sv[j][ch] = out ? s2[(size_t)ch * plane + (size_t)xe * H + y] : 0.f;
      fv[j] = out ? __ldg(row + xe) : 0;
    }
#pragma unroll
    for (int j = 0; j < kChunkH; ++j) {
      const int xe = x0 - j;
      if (xe < -E) break;
      float yo[2];
      az.step(r, cc[j], yo);
      if (yin && xe >= 0 && xe < Wd) {
        // demodulate: Re[e^{-i n w f} (filtered pair)]: Q_n for (cos, sin), P_n for the f-weighted pair
        const float2 cs = tab[fv[j]];
        pq[(size_t)xe * H + y] = dn * fmaf(cs.x, yo[0] + sv[j][0], cs.y * (yo[1] + sv[j][1]));
      }
    }
  }
}

// (P, Q) summed over the chunk's harmonics (and the earlier chunks' acc); the
// last chunk writes fhat = P / Q + T/2.  Block 32 x 32: threadIdx.x = row offset
// (coalesced reads of the transposed planes), tile transpose for the output.
__global__ void __launch_bounds__(1024) fbf_rec_out_kernel(const __grid_constant__ RecArgs r) {
  __shared__ float t[32][33];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int ty = threadIdx.y, tx = threadIdx.x;
  const int x = x0 + ty, y = y0 + tx;
  const int H = r.H, Wd = r.Wd;
  const bool in = x < Wd && y < H;
  float2 a = make_float2(0.f, 0.f);
  if (in) {
    const size_t o = (size_t)x * H + y, plane = (size_t)Wd * H;
    if (!r.first) a = r.acc[o];
    for (int nl = 0; nl < r.nh; ++nl) {
      a.x += r.pq[(size_t)(2 * nl) * plane + o];
      a.y += r.pq[(size_t)(2 * nl + 1) * plane + o];
    }
    if (!r.last) r.acc[o] = a;
  }
  if (!r.last) return;  // uniform over the grid
  t[ty][tx] = in ? a.x / a.y + r.c0 : 0.f;
  __syncthreads();
  const int ox = x0 + tx, oy = y0 + ty;  // write out[oy][ox] = t[tx][ty]: coalesced over tx
  if (ox < Wd && oy < H)
    *reinterpret_cast<float *>(reinterpret_cast<char *>(r.out) + (size_t)oy * r.out_pitch + (size_t)ox * sizeof(float)) =
        t[tx][ty];
}

}  // namespace

fbf_status launch_rec_u8(const FilterArgs &a, cudaStream_t s) {
  if (!a.rec || a.twoT < 2) return FBF_ERR_INVALID_ARGUMENT;
  const int H = a.H, Wd = a.Wd, K = a.K;
  if (H <= 0 || Wd <= 0) return FBF_OK;
  const size_t px = (size_t)H * Wd;
  const size_t per_h = px * (4 * sizeof(float) * 2 + sizeof(float2));  // vt, s2, pq
  constexpr size_t kBudget = (size_t)4 << 30;
  const int nh = (int)std::max<size_t>(1, std::min<size_t>((size_t)K, kBudget / per_h));
  const size_t vt_b = (size_t)nh * 4 * px * sizeof(float), pq_b = (size_t)nh * px * sizeof(float2);
  const size_t acc_b = K > nh ? px * sizeof(float2) : 0;
  char *scratch = nullptr;
  if (scratch_alloc(reinterpret_cast<void **>(&scratch), 2 * vt_b + pq_b + acc_b + 256, s) != FBF_OK)
    return FBF_ERR_CUDA;
  RecArgs r;
  r.in = static_cast<const unsigned char *>(a.in);
  r.in_pitch = a.in_pitch;
  r.out = a.out;
  r.out_pitch = a.out_pitch;
  r.H = H;
  r.Wd = Wd;
  r.twoT = a.twoT;
  r.border = a.border;
  r.E = a.rE;
  r.T = a.T;
  r.c0 = 0.5f * a.T;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      r.rn[i][j] = a.rn[i][j];
      r.rm[i][j] = a.rm[i][j];
      r.rp[i][j] = a.rp[i][j];
    }
  for (int k = 0; k < FBF_KMAX; ++k) r.d[k] = k < K ? a.d[k] : 0.f;
  r.vt = reinterpret_cast<float *>(scratch);
  r.s2 = reinterpret_cast<float *>(scratch + vt_b);
  r.pq = reinterpret_cast<float *>(scratch + 2 * vt_b);
  r.acc = acc_b ? reinterpret_cast<float2 *>(scratch + 2 * vt_b + pq_b) : nullptr;
  fbf_status st = FBF_OK;
  for (int n0 = 0; n0 < K && st == FBF_OK; n0 += nh) {
    r.n0 = n0;
    r.nh = std::min(nh, K - n0);
    r.first = n0 == 0;
    r.last = n0 + r.nh >= K;
    fbf_rec_v_kernel<<<dim3((Wd + 31) / 32, r.nh, 2), 32, 0, s>>>(r);
    fbf_rec_h_kernel<<<dim3((H + 31) / 32, r.nh, 2), 32, 0, s>>>(r);
    fbf_rec_out_kernel<<<dim3((Wd + 31) / 32, (H + 31) / 32), dim3(32, 32), 0, s>>>(r);
    st = cuda_status(cudaGetLastError());
  }
  if (scratch_free(scratch, s) != FBF_OK && st == FBF_OK) st = FBF_ERR_CUDA;
  return st;
}

}  // namespace fbf
