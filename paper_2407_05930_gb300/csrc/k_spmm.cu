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

// Vector of N consecutive T, aligned to its size up to 32 bytes (a 32-byte
// vector is one 256-bit access where the hardware has it, else two 16-byte ones).
template <typename T, int N>
struct alignas(sizeof(T) * N <= 32 ? sizeof(T) * N : 32) Vec {
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

// Thread layout.  A row is served by S = TPC * KL threads: TPC column
// threads (each owning CPT consecutive columns, TPC = C / CPT) times KL entry
// lanes (lane e takes the row's entries e, e + KL, ...).  The KL partial sums
// are combined with warp shuffles (S divides 32 when KL > 1), and entry lane 0
// runs the epilogue.  KL > 1 keeps several gathers of one row in flight, which
// is what hides the ptr -> idx -> X latency chain of short rows and spreads the
// long rows of the coarse levels over many lanes.
template <typename MT, typename XT, typename OT, int CPT, int KL, bool HAS_DOT, bool HAS_IFACE>
__global__ void __launch_bounds__(kBlock, 8) spmm_kernel(SpmmArgs a) {
  using CT = typename ComputeOf<MT, XT>::type;
  using DT = typename AccOf<XT>::type;  // per-thread dot partial type
  if (a.skip && *a.skip == 0) return;   // uniform over the grid
  const int C = a.C;
  const int TPC = C / CPT;
  const int S = TPC * KL;
  const int rows_pb = kBlock / S;
  const int g = threadIdx.x / S;
  const int w = threadIdx.x - g * S;
  const int e = KL > 1 ? w / TPC : 0;
  const int c0 = (w - e * TPC) * CPT;
  const bool slot_ok = g < rows_pb;
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

  // Grid-stride over row slots: a wave of blocks sweeps one contiguous window
  // of rows, so the far neighbours one block gathers were recently brought
  // into L2 by another.  The trip count is block-uniform (the shuffles need
  // every lane of the warp).
  for (int base = blockIdx.x * rows_pb; base < a.rows; base += gridDim.x * rows_pb) {
    const int row = base + g;
    const bool live = slot_ok && row < a.rows;
    CT acc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q] = (CT)0;
    if (live) {
      const int kb = __ldg(ptr + row), ke = __ldg(ptr + row + 1);
      int k = kb + e;
      for (; k + KL < ke; k += 2 * KL) {
        const int j0 = __ldg(idx + k), j1 = __ldg(idx + k + KL);
        const CT m0 = cvt<CT>(val[k]), m1 = cvt<CT>(val[k + KL]);
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
      if (HAS_IFACE && e == 0) {
        const uint32_t wd = __ldg(a.imask + (row >> 5));
        const uint32_t bit = 1u << (row & 31);
        if (wd & bit) {
          const int f = __ldg(a.iprefix + (row >> 5)) + __popc(wd & (bit - 1u));
          const CT* __restrict__ iv = static_cast<const CT*>(a.ival);
          for (int ee = __ldg(a.iptr + f); ee < __ldg(a.iptr + f + 1); ++ee) {
            const int j = __ldg(a.icol + ee);
            const Vec<XT, CPT> xv = ldv<XT, CPT>(X + (int64_t)j * C + c0);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
              const int blk = (c0 + q) % a.nb;
              acc[q] = fma(iv[(int64_t)ee * a.nb + blk], (CT)xv.v[q], acc[q]);
            }
          }
        }
      }
    }
    if (KL > 1) {
#pragma unroll
      for (int off = KL / 2; off >= 1; off >>= 1) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off * TPC);
      }
    }
    if (live && e == 0) {
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
    extern __shared__ double sm[];
    double part[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) part[q] = (slot_ok && e == 0) ? (double)dpart[q] : 0.0;
    block_dot<CPT>(a.dot, part, c0, slot_ok && e == 0, g, rows_pb, S, C, sm);
  }
}

template <typename MT, typename XT, typename OT, int CPT, int KL>
static void launch_k(const SpmmArgs& a, cudaStream_t st) {
  const int TPC = a.C / CPT;
  const int rows_pb = kBlock / (TPC * KL);
  int64_t need = ((int64_t)a.rows + rows_pb - 1) / rows_pb;
  int grid = (int)std::min<int64_t>(need, (int64_t)max_grid_blocks());
  if (grid < 1) grid = 1;
  const bool dot = a.dot.mode != DOT_NONE;
  const bool ifc = a.imask != nullptr;
  count_launch();
  // one full wave of resident blocks (the register count differs per variant)
  auto run = [&](auto kern, size_t smem) {
    int g = std::min(grid, resident_grid((const void*)kern, smem));
    if (dot && (int64_t)g * a.C > a.dot.sc.partial_cap) g = (int)(a.dot.sc.partial_cap / a.C);
    kern<<<g, kBlock, smem, st>>>(a);
  };
  if (dot) {
    const size_t smem = sizeof(double) * (size_t)dot_smem_doubles(TPC * KL, rows_pb, a.C);
    if (ifc)
      run(spmm_kernel<MT, XT, OT, CPT, KL, true, true>, smem);
    else
      run(spmm_kernel<MT, XT, OT, CPT, KL, true, false>, smem);
  } else {
    if (ifc)
      run(spmm_kernel<MT, XT, OT, CPT, KL, false, true>, 0);
    else
      run(spmm_kernel<MT, XT, OT, CPT, KL, false, false>, 0);
  }
}

template <typename MT, typename XT, typename OT, int CPT>
static void launch_t(const SpmmArgs& a, cudaStream_t st) {
  const int TPC = a.C / CPT;
  // entry lanes: only with a power-of-two column-thread count, and S <= 32
  int kl = a.kl > 0 ? a.kl : 1;
  if (TPC & (TPC - 1)) kl = 1;
  while (kl > 1 && TPC * kl > 32) kl >>= 1;
  switch (kl) {
    case 1: launch_k<MT, XT, OT, CPT, 1>(a, st); break;
    case 2: launch_k<MT, XT, OT, CPT, 2>(a, st); break;
    case 4: launch_k<MT, XT, OT, CPT, 4>(a, st); break;
    case 8: launch_k<MT, XT, OT, CPT, 8>(a, st); break;
    default: launch_k<MT, XT, OT, CPT, 16>(a, st); break;
  }
}

template <typename MT, typename XT, typename OT>
static void launch_c(const SpmmArgs& a, cudaStream_t st) {
  // V: elements of the narrower of X / Y in one 16-byte vector
  constexpr int V = 16 / (int)sizeof(XT) < 16 / (int)sizeof(OT) ? 16 / (int)sizeof(XT) : 16 / (int)sizeof(OT);
  const int want = a.cpt > 0 ? a.cpt : V;
  if (want >= 2 * V && V == 4 && a.C % 8 == 0 && a.C / 8 <= kBlock)
    launch_t<MT, XT, OT, 8>(a, st);
  else if (want >= 2 * V && V == 2 && a.C % 4 == 0 && a.C / 4 <= kBlock)
    launch_t<MT, XT, OT, 4>(a, st);
  else if (V >= 4 && a.C % 4 == 0 && a.C / 4 <= kBlock)
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
