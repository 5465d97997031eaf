// Device helpers shared by the filter kernels: border mapping and staging of
// an image tile plus its halo into shared memory.
#pragma once

#include <cuda_runtime.h>

#include "fbf.h"

namespace fbf {

// Half-sample symmetric reflection into [0, n): ... 1 0 | 0 1 ... n-1 | n-1 ...
__device__ __forceinline__ int reflect_index(int i, int n) {
  if (i >= 0 && i < n) return i;
  const int p = 2 * n;
  int m = i % p;
  if (m < 0) m += p;
  return m < n ? m : p - 1 - m;
}

// Stage the halo tile whose ext pixel (0, 0) is image pixel (y0, x0) into
// tileT[ex * sx + ey * sy], for ey < nrows and ex < ncols <= 32 * CG.  Each
// entry is (pixel value) * scale -- the byte offset of that value's row in a
// channel table -- or `sentinel` for padding (ey >= rows_valid or ex >=
// cols_valid) and, under TRUNCATE, for pixels outside the image.  Warps take
// rows, lanes take columns (coalesced global reads; column-major writes, sy = 1,
// hit distinct banks when sx / 2 is odd); up to 8 loads per thread are in flight.
template <int NT, int CG = 4>
__device__ __forceinline__ void stage_tile(const unsigned char *__restrict__ in, size_t pitch, int H, int Wd,
                                           int border, int y0, int x0, int rows_valid, int cols_valid,
                                           int nrows, int ncols, unsigned short *tileT, int sx, int sy,
                                           unsigned short scale, unsigned short sentinel) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool reflect = border == FBF_BORDER_REFLECT;
  for (int ey0 = warp; ey0 < nrows; ey0 += 2 * NW) {
    unsigned short v[2][CG];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int ey = ey0 + rr * NW;
      int iy = y0 + ey;
      bool row_ok = ey < nrows && ey < rows_valid;
      if (reflect)
        iy = reflect_index(iy, H);
      else
        row_ok = row_ok && iy >= 0 && iy < H;
      const unsigned char *rowp = in + (size_t)(row_ok ? iy : 0) * pitch;
#pragma unroll
      for (int k = 0; k < CG; ++k) {
        const int ex = lane + 32 * k;
        int ix = x0 + ex;
        bool ok = row_ok && ex < cols_valid;
        if (reflect)
          ix = reflect_index(ix, Wd);
        else
          ok = ok && ix >= 0 && ix < Wd;
        v[rr][k] = ok ? (unsigned short)(__ldg(rowp + ix) * scale) : sentinel;
      }
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int ey = ey0 + rr * NW;
      if (ey < nrows) {
#pragma unroll
        for (int k = 0; k < CG; ++k) {
          const int ex = lane + 32 * k;
          if (ex < ncols) tileT[ex * sx + ey * sy] = v[rr][k];
        }
      }
    }
  }
}

}  // namespace fbf
