// Dense coarsest-level solve (Sec. 5: a direct method on the coarsest level)
// shared by the stand-alone kernel and the persistent coarse-cycle kernel, so
// both give the same bits: Z = A_c^{-1} Y with the precomputed FP64 inverse,
// FP64 arithmetic.
#pragma once

#include <cstdint>

namespace amgsym {

// Rows i = warp, warp + nwarps, ... of Z (n x C) by whole warps: lane l sums
// the terms j = l, l + 32, ... in ascending order for 8 columns at a time
// (the inverse's row read once per 8 columns, coalesced across the lanes;
// the lanes' rows of Y contiguous), then a fixed butterfly over the lanes
// (xor 16, 8, 4, 2, 1) combines the 32 partial sums and lane 0 stores them.
// LD(p) loads one Y value (through L2 when Y was written in the same launch).
template <typename T, typename LD>
__device__ __forceinline__ void coarse_rows_warp(int32_t n, int32_t C, const double* __restrict__ Ainv,
                                                 const T* Y, T* Z, int64_t warp, int64_t nwarps, LD ld) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* a = Ainv + i * n;
    for (int c0 = 0; c0 < C; c0 += 8) {
      const int nc = C - c0 < 8 ? C - c0 : 8;
      double acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0;
      // four terms per lane in flight (all loads first, then the fmas in
      // ascending j: the same sum as one term at a time)
      int j = lane;
      for (; j + 96 < n; j += 128) {
        double av[4];
        double yv[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = a[j + 32 * u];
          const T* y = Y + (int64_t)(j + 32 * u) * C + c0;
#pragma unroll
          for (int q = 0; q < 8; ++q) yv[u][q] = q < nc ? (double)ld(y + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < nc) acc[q] = fma(av[u], yv[u][q], acc[q]);
        }
      }
      for (; j < n; j += 32) {
        const double av = a[j];
        const T* y = Y + (int64_t)j * C + c0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nc) acc[q] = fma(av, (double)ld(y + q), acc[q]);
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
      }
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nc) Z[i * C + c0 + q] = (T)acc[q];
      }
    }
  }
}

}  // namespace amgsym
