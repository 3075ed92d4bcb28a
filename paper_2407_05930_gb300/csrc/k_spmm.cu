// Sparse matrix times interleaved multi-vector (SpMM) with fused epilogues.
//
// One kernel serves every sparse product of the solve:
//   * the reduced operator Y = (I (x) A_inn + blockdiag(A_out,i)) X of
//     eq. "hL_splitting": A_inn is read once for all c = nrhs * 2^s columns
//     (eq. "spmm": the SpMM form of Sec. 2 that raises arithmetic intensity
//     by 2^s), and the interface correction is added in the same pass (the
//     paper's fused SpMM + interface SpMV + linear combination, Sec. 2);
//   * the V-cycle products with A_l, G_l, G_l^T, R_l = P_l^T and P_l
//     (Alg. "apply" shape, Sec. 3.2), with epilogues for residuals
//     (Y = Z - A X) and updates (Y = Z + w G^T X).
//
// Layout: X, Y, Z are [rows][C] row-major; thread t of a 256-thread block
// owns columns c0 = (t % TPR) * CPT .. c0 + CPT - 1 of row slot t / TPR,
// TPR = C / CPT, so one 16-byte vector load fetches a thread's columns of a
// neighbour row and the TPR threads of a row read each matrix entry once
// (broadcast).  Rows are walked grid-stride so a wave of blocks touches a
// contiguous window of rows (L2 reuse of the gathered X rows).
//
// Epilogue: Y = alpha * (M X) + beta * Z (Z read only when beta != 0), then
// an optional per-column dot (W.Y or Y.Y) reduced deterministically.
#include <cuda_bf16.h>

#include "device.h"
#include "dot.cuh"

namespace amgsym {

template <typename T>
struct AccOf {
  using type = float;
};
template <>
struct AccOf<double> {
  using type = double;
};

template <typename T>
__device__ __forceinline__ float to_f(T v) {
  return (float)v;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename A, typename T>
__device__ __forceinline__ A cvt(T v) {
  return (A)v;
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

// Vector of N consecutive T (N * sizeof(T) <= 16 bytes, naturally aligned).
template <typename T, int N>
struct alignas(sizeof(T) * N) Vec {
  T v[N];
};

template <typename T, int N>
__device__ __forceinline__ Vec<T, N> ldv(const T* p) {
  return *reinterpret_cast<const Vec<T, N>*>(p);
}
template <typename T, int N>
__device__ __forceinline__ Vec<T, N> ldv_stream(const T* p) {
  return __ldcs(reinterpret_cast<const Vec<T, N>*>(p));
}
template <typename T, int N>
__device__ __forceinline__ void stv(T* p, const Vec<T, N>& v) {
  *reinterpret_cast<Vec<T, N>*>(p) = v;
}

// The compute type: FP64 if either operand is FP64, else FP32.
template <typename MT, typename XT>
struct ComputeOf {
  using type = float;
};
template <typename XT>
struct ComputeOf<double, XT> {
  using type = double;
};
template <typename MT>
struct ComputeOf<MT, double> {
  using type = double;
};
template <>
struct ComputeOf<double, double> {
  using type = double;
};

template <typename MT, typename XT, typename OT, int CPT, bool HAS_DOT, bool HAS_IFACE>
__global__ void __launch_bounds__(kBlock) spmm_kernel(SpmmArgs a) {
  using CT = typename ComputeOf<MT, XT>::type;
  using DT = typename AccOf<XT>::type;  // per-thread dot partial type
  if (a.skip && *a.skip == 0) return;  // uniform over the grid
  const int C = a.C;
  const int TPR = C / CPT;
  const int rows_pb = kBlock / TPR;
  const int rloc = threadIdx.x / TPR;
  const int c0 = (threadIdx.x % TPR) * CPT;
  const bool has_cols = rloc < rows_pb;
  const MT* __restrict__ val = static_cast<const MT*>(a.val);
  const XT* __restrict__ X = static_cast<const XT*>(a.X);
  // Y may alias Z (in-place update z += ...); each row reads Z before writing Y.
  const XT* Z = static_cast<const XT*>(a.Z);
  OT* Y = static_cast<OT*>(a.Y);
  const int32_t* __restrict__ ptr = a.ptr;
  const int32_t* __restrict__ idx = a.idx;
  const CT alpha = (CT)a.alpha, beta = (CT)a.beta;
  DT dpart[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) dpart[q] = (DT)0;

  if (has_cols) {
    for (int row = blockIdx.x * rows_pb + rloc; row < a.rows; row += gridDim.x * rows_pb) {
      CT acc[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = (CT)0;
      const int kb = __ldg(ptr + row), ke = __ldg(ptr + row + 1);
      int k = kb;
      // two entries per step for memory-level parallelism
      for (; k + 1 < ke; k += 2) {
        const int j0 = __ldg(idx + k), j1 = __ldg(idx + k + 1);
        const CT m0 = cvt<CT>(val[k]), m1 = cvt<CT>(val[k + 1]);
        const Vec<XT, CPT> x0 = ldv<XT, CPT>(X + (int64_t)j0 * C + c0);
        const Vec<XT, CPT> x1 = ldv<XT, CPT>(X + (int64_t)j1 * C + c0);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          acc[q] = fma(m0, (CT)x0.v[q], acc[q]);
          acc[q] = fma(m1, (CT)x1.v[q], acc[q]);
        }
      }
      if (k < ke) {
        const int j0 = __ldg(idx + k);
        const CT m0 = cvt<CT>(val[k]);
        const Vec<XT, CPT> x0 = ldv<XT, CPT>(X + (int64_t)j0 * C + c0);
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = fma(m0, (CT)x0.v[q], acc[q]);
      }
      if (HAS_IFACE) {
        const uint32_t w = __ldg(a.imask + (row >> 5));
        const uint32_t bit = 1u << (row & 31);
        if (w & bit) {
          const int f = __ldg(a.iprefix + (row >> 5)) + __popc(w & (bit - 1u));
          const CT* __restrict__ iv = static_cast<const CT*>(a.ival);
          for (int e = __ldg(a.iptr + f); e < __ldg(a.iptr + f + 1); ++e) {
            const int j = __ldg(a.icol + e);
            const Vec<XT, CPT> xv = ldv<XT, CPT>(X + (int64_t)j * C + c0);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
              const int blk = (c0 + q) % a.nb;
              acc[q] = fma(iv[(int64_t)e * a.nb + blk], (CT)xv.v[q], acc[q]);
            }
          }
        }
      }
      Vec<OT, CPT> out;
      if (a.beta != 0.0) {
        const Vec<XT, CPT> zv = ldv<XT, CPT>(Z + (int64_t)row * C + c0);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const CT y = alpha * acc[q] + beta * (CT)zv.v[q];
          out.v[q] = (OT)y;
          acc[q] = y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const CT y = alpha * acc[q];
          out.v[q] = (OT)y;
          acc[q] = y;
        }
      }
      stv<OT, CPT>(Y + (int64_t)row * C + c0, out);
      if (HAS_DOT) {
        if (a.dot.mode == DOT_WY) {
          const Vec<XT, CPT> wv = ldv<XT, CPT>(static_cast<const XT*>(a.dot.W) + (int64_t)row * C + c0);
#pragma unroll
          for (int q = 0; q < CPT; ++q) dpart[q] += (DT)wv.v[q] * (DT)acc[q];
        } else {
#pragma unroll
          for (int q = 0; q < CPT; ++q) dpart[q] += (DT)acc[q] * (DT)acc[q];
        }
      }
    }
  }
  if (HAS_DOT) {
    __shared__ double sm[kBlock * CPT + 2 * kBlock];
    double part[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) part[q] = (double)dpart[q];
    block_dot<CPT>(a.dot, part, c0, has_cols, rloc, rows_pb, C, sm);
  }
}

template <typename MT, typename XT, typename OT, int CPT>
static void launch_t(const SpmmArgs& a, cudaStream_t st) {
  const int TPR = a.C / CPT;
  const int rows_pb = kBlock / TPR;
  int64_t need = ((int64_t)a.rows + rows_pb - 1) / rows_pb;
  int grid = (int)std::min<int64_t>(need, (int64_t)max_grid_blocks());
  if (grid < 1) grid = 1;
  const bool dot = a.dot.mode != DOT_NONE;
  const bool ifc = a.imask != nullptr;
  count_launch();
  if (dot) {
    if ((int64_t)grid * a.C > a.dot.sc.partial_cap) grid = (int)(a.dot.sc.partial_cap / a.C);
    if (ifc)
      spmm_kernel<MT, XT, OT, CPT, true, true><<<grid, kBlock, 0, st>>>(a);
    else
      spmm_kernel<MT, XT, OT, CPT, true, false><<<grid, kBlock, 0, st>>>(a);
  } else {
    if (ifc)
      spmm_kernel<MT, XT, OT, CPT, false, true><<<grid, kBlock, 0, st>>>(a);
    else
      spmm_kernel<MT, XT, OT, CPT, false, false><<<grid, kBlock, 0, st>>>(a);
  }
}

template <typename MT, typename XT, typename OT>
static void launch_c(const SpmmArgs& a, cudaStream_t st) {
  constexpr int V = 16 / (int)sizeof(XT) < 16 / (int)sizeof(OT) ? 16 / (int)sizeof(XT) : 16 / (int)sizeof(OT);
  if (V >= 4 && a.C % 4 == 0 && a.C / 4 <= kBlock)
    launch_t<MT, XT, OT, 4>(a, st);
  else if (V >= 2 && a.C % 2 == 0 && a.C / 2 <= kBlock)
    launch_t<MT, XT, OT, 2>(a, st);
  else
    launch_t<MT, XT, OT, 1>(a, st);
}

void launch_spmm(ValType mt, VecType xt, VecType ot, const SpmmArgs& a, cudaStream_t st) {
  if (a.rows <= 0) return;
  if (mt == VAL_F64 && xt == VEC_F64 && ot == VEC_F64)
    launch_c<double, double, double>(a, st);
  else if (mt == VAL_F64 && xt == VEC_F64 && ot == VEC_F32)
    launch_c<double, double, float>(a, st);
  else if (mt == VAL_F32 && xt == VEC_F32 && ot == VEC_F32)
    launch_c<float, float, float>(a, st);
  else if (mt == VAL_BF16 && xt == VEC_F32 && ot == VEC_F32)
    launch_c<__nv_bfloat16, float, float>(a, st);
  else
    fail(AMGSYM_ERR_ARG, "unsupported SpMM precision combination");
}

}  // namespace amgsym
