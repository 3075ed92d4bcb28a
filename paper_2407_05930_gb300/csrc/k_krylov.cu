// Multi-vector kernels of the GMRES solve and of the low-rank correction
// (LRCAMG, Sec. 2.2): dots of one vector with many, sums of many vectors with
// per-column coefficients, per-column scaling.  FP64, interleaved [rows][C]
// layouts.  A "vector set" V holds J vectors of rows x Cv values, vector j at
// V + j * vstride; column c of a [rows][C] vector pairs with column c % Cv of
// the set (Cv = C for GMRES bases, Cv = 2^s for per-block correction vectors
// shared by every right-hand side).  Sums run in a fixed order (per-thread
// rows, then a fixed combination across threads and blocks): results are
// bit-reproducible run to run.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.h"
#include "dot.cuh"

namespace amgsym {

namespace {

constexpr int kJChunk = 8;  // vectors of a set per pass over W

// part[(blk * J + j) * C + c] = sum over this block's rows of V_j[row][c % Cv] * W[row][c].
__global__ void __launch_bounds__(kBlock) mdot_partial_kernel(const double* __restrict__ V, int64_t vstride,
                                                              int32_t Cv, int32_t J, const double* __restrict__ W,
                                                              int64_t rows, int32_t C, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const int rpb = kBlock / C;  // rows per block step
  const int col = threadIdx.x % C, rl = threadIdx.x / C;
  const bool act = rl < rpb;
  const int vc = col % Cv;
  for (int j0 = 0; j0 < J; j0 += kJChunk) {
    double acc[kJChunk];
#pragma unroll
    for (int u = 0; u < kJChunk; ++u) acc[u] = 0.0;
    if (act) {
      for (int64_t row = blockIdx.x * (int64_t)rpb + rl; row < rows; row += (int64_t)gridDim.x * rpb) {
        const double w = W[row * C + col];
#pragma unroll
        for (int u = 0; u < kJChunk; ++u)
          if (j0 + u < J) acc[u] = fma(V[(int64_t)(j0 + u) * vstride + row * Cv + vc], w, acc[u]);
      }
    }
    for (int u = 0; u < kJChunk && j0 + u < J; ++u) {
      sm[threadIdx.x] = acc[u];
      __syncthreads();
      if (threadIdx.x < C) {
        double s = 0.0;
        for (int r = 0; r < rpb; ++r) s += sm[r * C + threadIdx.x];
        part[((int64_t)blockIdx.x * J + j0 + u) * C + threadIdx.x] = s;
      }
      __syncthreads();
    }
  }
}

// H[j * C + c] = sum over blocks (in block order) of the partials.
__global__ void mdot_final_kernel(const double* __restrict__ part, int32_t nblk, int32_t J, int32_t C,
                                  double* __restrict__ H) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < J * C; t += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * J * C + t];
    H[t] = s;
  }
}

// W[row][c] += sign * sum_j V_j[row][c % Cv] * H[j * C + c]  (j in order).
__global__ void __launch_bounds__(kBlock) maxpy_kernel(const double* __restrict__ V, int64_t vstride, int32_t Cv,
                                                       int32_t J, const double* __restrict__ H, double sign,
                                                       double* __restrict__ W, int64_t rows, int32_t C) {
  const int64_t total = rows * C;
  for (int64_t e = blockIdx.x * (int64_t)kBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kBlock) {
    const int64_t row = e / C;
    const int c = (int)(e - row * C);
    const int64_t vo = row * Cv + c % Cv;
    double acc = 0.0;
    for (int j = 0; j < J; ++j) acc = fma(V[(int64_t)j * vstride + vo], H[j * C + c], acc);
    W[e] = fma(sign, acc, W[e]);
  }
}

// Out[row][c] = W[row][c] * s[c].
__global__ void __launch_bounds__(kBlock) colscale_kernel(const double* __restrict__ W, const double* __restrict__ s,
                                                          double* __restrict__ out, int64_t rows, int32_t C) {
  const int64_t total = rows * C;
  for (int64_t e = blockIdx.x * (int64_t)kBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kBlock)
    out[e] = W[e] * s[e % C];
}

int grid_elems(int64_t total) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + kBlock - 1) / kBlock, max_grid_blocks()));
}

}  // namespace

int mdot_blocks(int64_t rows, int32_t C) {
  const int rpb = kBlock / C;
  return (int)std::max<int64_t>(1, std::min<int64_t>((rows + rpb - 1) / rpb, num_sms() * 4));
}

void launch_mdot(const double* V, int64_t vstride, int32_t Cv, int32_t J, const double* W, int64_t rows, int32_t C,
                 double* part, double* H, cudaStream_t st) {
  if (J <= 0) return;
  const int g = mdot_blocks(rows, C);
  count_launch(2);
  mdot_partial_kernel<<<g, kBlock, 0, st>>>(V, vstride, Cv, J, W, rows, C, part);
  mdot_final_kernel<<<std::max(1, (J * C + 255) / 256), 256, 0, st>>>(part, g, J, C, H);
}

void launch_maxpy(const double* V, int64_t vstride, int32_t Cv, int32_t J, const double* H, double sign, double* W,
                  int64_t rows, int32_t C, cudaStream_t st) {
  if (J <= 0) return;
  count_launch();
  maxpy_kernel<<<grid_elems(rows * C), kBlock, 0, st>>>(V, vstride, Cv, J, H, sign, W, rows, C);
}

void launch_colscale(const double* W, const double* s, double* out, int64_t rows, int32_t C, cudaStream_t st) {
  count_launch();
  colscale_kernel<<<grid_elems(rows * C), kBlock, 0, st>>>(W, s, out, rows, C);
}

}  // namespace amgsym
