// Batched kernels: one launch serves many independent problems.
//
// Each launch walks a work list of items (a row range of one problem's
// operation); the grid is one full wave of resident blocks and every block
// takes items blockIdx.x, blockIdx.x + gridDim.x, ... (a persistent work-list
// kernel).  A block copies the item's argument record to shared memory and
// runs the same tile code as the single-problem kernels, so a batch of
// uneven problems costs one launch per step of the V-cycle / PCG instead of
// one per problem.  Dot products are reduced per problem: each item writes
// one partial per column and the last item of a problem (integer ticket)
// finalises that problem's CG scalars, in a fixed order.
#include <cuda_bf16.h>

#include <algorithm>

#include "spmm_common.cuh"

namespace amgsym {

template <typename MT, typename XT, typename OT, int CPT, int KL, bool HAS_DOT, bool HAS_IFACE, bool DIA>
__global__ void __launch_bounds__(kBlock, 4)
    spmm_batch_kernel(const SpmmArgs* __restrict__ args, const BItem* __restrict__ items, int32_t n_items,
                      const BDot* __restrict__ dots) {
  using DT = typename AccOf<XT>::type;
  __shared__ __align__(16) unsigned char sa_raw[sizeof(SpmmArgs)];
  SpmmArgs& a = *reinterpret_cast<SpmmArgs*>(sa_raw);
  extern __shared__ double sm[];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const BItem bi = items[it];
    __syncthreads();  // the previous item is done with the record
    if (threadIdx.x == 0) a = args[bi.arg];
    __syncthreads();
    if (a.skip && *a.skip == 0) continue;  // block-uniform
    DT dpart[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) dpart[q] = (DT)0;
    spmm_tile<MT, XT, OT, CPT, KL, HAS_DOT, HAS_IFACE, DIA>(a, bi.first_slot, 1, bi.row_end, dpart, false);
    if (HAS_DOT) {
      const TileLayout t = tile_layout<CPT, KL>(a.C);
      double part[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) part[q] = (t.slot_ok && t.e == 0) ? (double)dpart[q] : 0.0;
      const BDot bd = dots[bi.arg];
      block_dot2<CPT>(a.dot, part, t.c0, t.slot_ok && t.e == 0, t.g, t.rows_pb, t.S, a.C, sm, bi.slot, bd);
    }
  }
}

template <typename MT, typename XT, typename OT, int CPT, int KL, bool DIA = false>
static void spmm_batch_k(bool dot, bool iface, const SpmmArgs* args, const BItem* items, int32_t n_items,
                         const BDot* dots, size_t smem, cudaStream_t st) {
  auto run = [&](auto kern) {
    const int g = std::max(1, std::min<int>(n_items, resident_grid((const void*)kern, smem)));
    kern<<<g, kBlock, smem, st>>>(args, items, n_items, dots);
  };
  if (dot) {
    if (iface)
      run(spmm_batch_kernel<MT, XT, OT, CPT, KL, true, true, DIA>);
    else
      run(spmm_batch_kernel<MT, XT, OT, CPT, KL, true, false, DIA>);
  } else {
    if (iface)
      run(spmm_batch_kernel<MT, XT, OT, CPT, KL, false, true, DIA>);
    else
      run(spmm_batch_kernel<MT, XT, OT, CPT, KL, false, false, DIA>);
  }
}

// dia: every record of the launch is in the diagonal-offset form (one lane per row)
template <typename MT, typename XT, typename OT, int CPT>
static void spmm_batch_c(int kl, bool dot, bool iface, bool dia, const SpmmArgs* args, const BItem* items,
                         int32_t n_items, const BDot* dots, size_t smem, cudaStream_t st) {
  if (dia) {
    spmm_batch_k<MT, XT, OT, CPT, 1, true>(dot, iface, args, items, n_items, dots, smem, st);
    return;
  }
  switch (kl) {
    case 1: spmm_batch_k<MT, XT, OT, CPT, 1>(dot, iface, args, items, n_items, dots, smem, st); break;
    case 2: spmm_batch_k<MT, XT, OT, CPT, 2>(dot, iface, args, items, n_items, dots, smem, st); break;
    case 4: spmm_batch_k<MT, XT, OT, CPT, 4>(dot, iface, args, items, n_items, dots, smem, st); break;
    case 8: spmm_batch_k<MT, XT, OT, CPT, 8>(dot, iface, args, items, n_items, dots, smem, st); break;
    default: spmm_batch_k<MT, XT, OT, CPT, 16>(dot, iface, args, items, n_items, dots, smem, st); break;
  }
}

template <typename MT, typename XT, typename OT>
static void spmm_batch_t(int cpt, int kl, bool dot, bool iface, bool dia, const SpmmArgs* args, const BItem* items,
                         int32_t n_items, const BDot* dots, size_t smem, cudaStream_t st) {
  switch (cpt) {
    case 8: spmm_batch_c<MT, XT, OT, 8>(kl, dot, iface, dia, args, items, n_items, dots, smem, st); break;
    case 4: spmm_batch_c<MT, XT, OT, 4>(kl, dot, iface, dia, args, items, n_items, dots, smem, st); break;
    case 2: spmm_batch_c<MT, XT, OT, 2>(kl, dot, iface, dia, args, items, n_items, dots, smem, st); break;
    default: spmm_batch_c<MT, XT, OT, 1>(kl, dot, iface, dia, args, items, n_items, dots, smem, st); break;
  }
}

void launch_spmm_batch(ValType mt, VecType xt, VecType ot, int cpt, int kl, bool dot, bool iface, bool dia,
                       const SpmmArgs* args, const BItem* items, int32_t n_items, const BDot* dots, size_t smem,
                       cudaStream_t st) {
  if (n_items <= 0) return;
  count_launch();
  if (mt == VAL_F32 && xt == VEC_F32 && ot == VEC_F32)
    spmm_batch_t<float, float, float>(cpt, kl, dot, iface, dia, args, items, n_items, dots, smem, st);
  else if (mt == VAL_BF16 && xt == VEC_F32 && ot == VEC_F32)
    spmm_batch_t<__nv_bfloat16, float, float>(cpt, kl, dot, iface, dia, args, items, n_items, dots, smem, st);
  else if (mt == VAL_F64 && xt == VEC_F64 && ot == VEC_F32)
    spmm_batch_t<double, double, float>(cpt <= 2 ? cpt : 2, kl, dot, iface, dia, args, items, n_items, dots, smem,
                                        st);
  else if (mt == VAL_F64 && xt == VEC_F64 && ot == VEC_F64)
    spmm_batch_t<double, double, double>(cpt <= 4 ? cpt : 4, kl, dot, iface, dia, args, items, n_items, dots, smem,
                                         st);
  else
    fail(AMGSYM_ERR_ARG, "unsupported batched SpMM precision combination");
}

// ---------------------------------------------------------------------------
// Batched PCG vector steps (update1 with its convergence dot, update2, copy).

template <typename T, int N>
struct alignas(sizeof(T) * N <= 32 ? sizeof(T) * N : 32) VecB {
  T v[N];
};

template <typename T, int CPT, int OP>
__global__ void __launch_bounds__(kBlock) vec_batch_kernel(const UpdArgs* __restrict__ args,
                                                          const BItem* __restrict__ items, int32_t n_items,
                                                          const BDot* __restrict__ dots) {
  using DT = typename AccOf<T>::type;
  using V = VecB<T, CPT>;
  __shared__ __align__(16) unsigned char ua_raw[sizeof(UpdArgs)];
  UpdArgs& a = *reinterpret_cast<UpdArgs*>(ua_raw);
  extern __shared__ double sm[];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const BItem bi = items[it];
    __syncthreads();
    if (threadIdx.x == 0) a = args[bi.arg];
    __syncthreads();
    if (a.skip && *a.skip == 0) continue;
    const int C = a.C;
    const int TPR = C / CPT;
    const int rows_pb = kBlock / TPR;
    const int rloc = threadIdx.x / TPR;
    const int c0 = (threadIdx.x % TPR) * CPT;
    const bool has_cols = rloc < rows_pb;
    DT part[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) part[k] = (DT)0;
    if (has_cols) {
      if (OP == BOP_UPDATE1) {
        T al[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) al[k] = (T)a.dot.sc.alpha[c0 + k];
        T* x = static_cast<T*>(a.x);
        T* r = static_cast<T*>(a.r);
        const T* p = static_cast<const T*>(a.p);
        const T* q = static_cast<const T*>(a.q);
        for (int64_t row = (int64_t)bi.first_slot * rows_pb + rloc; row < bi.row_end; row += rows_pb) {
          const int64_t o = row * C + c0;
          V xv = *reinterpret_cast<const V*>(x + o);
          V rv = *reinterpret_cast<const V*>(r + o);
          const V pv = *reinterpret_cast<const V*>(p + o);
          const V qv = *reinterpret_cast<const V*>(q + o);
#pragma unroll
          for (int k = 0; k < CPT; ++k) {
            xv.v[k] = xv.v[k] + al[k] * pv.v[k];
            rv.v[k] = rv.v[k] - al[k] * qv.v[k];
            part[k] += (DT)rv.v[k] * (DT)rv.v[k];
          }
          *reinterpret_cast<V*>(x + o) = xv;
          *reinterpret_cast<V*>(r + o) = rv;
        }
      } else if (OP == BOP_UPDATE2) {
        T b[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) b[k] = (T)a.beta[c0 + k];
        T* p = static_cast<T*>(a.x);
        const T* z = static_cast<const T*>(a.p);
        for (int64_t row = (int64_t)bi.first_slot * rows_pb + rloc; row < bi.row_end; row += rows_pb) {
          const int64_t o = row * C + c0;
          V pv = *reinterpret_cast<const V*>(p + o);
          const V zv = *reinterpret_cast<const V*>(z + o);
#pragma unroll
          for (int k = 0; k < CPT; ++k) pv.v[k] = zv.v[k] + b[k] * pv.v[k];
          *reinterpret_cast<V*>(p + o) = pv;
        }
      } else if (OP == BOP_JACOBI) {
        // the diagonal smoother step of the stand-alone jacobi kernel
        T* z = static_cast<T*>(a.x);
        const T* src = static_cast<const T*>(a.p);
        const T* jd = static_cast<const T*>(a.jd);
        for (int64_t row = (int64_t)bi.first_slot * rows_pb + rloc; row < bi.row_end; row += rows_pb) {
          const int64_t o = row * C + c0;
          const T d = jd[row];
          const V sv = *reinterpret_cast<const V*>(src + o);
          V zv;
          if (a.accumulate) {
            zv = *reinterpret_cast<const V*>(z + o);
#pragma unroll
            for (int k = 0; k < CPT; ++k) zv.v[k] = fma(d, sv.v[k], zv.v[k]);
          } else {
#pragma unroll
            for (int k = 0; k < CPT; ++k) zv.v[k] = d * sv.v[k];
          }
          *reinterpret_cast<V*>(z + o) = zv;
        }
      } else {
        T* d = static_cast<T*>(a.x);
        const T* s = static_cast<const T*>(a.p);
        for (int64_t row = (int64_t)bi.first_slot * rows_pb + rloc; row < bi.row_end; row += rows_pb) {
          const int64_t o = row * C + c0;
          *reinterpret_cast<V*>(d + o) = *reinterpret_cast<const V*>(s + o);
        }
      }
    }
    if (OP == BOP_UPDATE1) {
      double pd[CPT];
#pragma unroll
      for (int k = 0; k < CPT; ++k) pd[k] = has_cols ? (double)part[k] : 0.0;
      const BDot bd = dots[bi.arg];
      block_dot2<CPT>(a.dot, pd, c0, has_cols, rloc, rows_pb, TPR, C, sm, bi.slot, bd);
    }
  }
}

template <typename T, int CPT>
static void vec_batch_c(int op, const UpdArgs* args, const BItem* items, int32_t n_items, const BDot* dots,
                        size_t smem, cudaStream_t st) {
  auto run = [&](auto kern) {
    const int g = std::max(1, std::min<int>(n_items, resident_grid((const void*)kern, smem)));
    kern<<<g, kBlock, smem, st>>>(args, items, n_items, dots);
  };
  if (op == BOP_UPDATE1)
    run(vec_batch_kernel<T, CPT, BOP_UPDATE1>);
  else if (op == BOP_UPDATE2)
    run(vec_batch_kernel<T, CPT, BOP_UPDATE2>);
  else if (op == BOP_JACOBI)
    run(vec_batch_kernel<T, CPT, BOP_JACOBI>);
  else
    run(vec_batch_kernel<T, CPT, BOP_COPY>);
}

void launch_vec_batch(int op, VecType vt, int cpt, const UpdArgs* args, const BItem* items, int32_t n_items,
                      const BDot* dots, size_t smem, cudaStream_t st) {
  if (n_items <= 0) return;
  count_launch();
  if (vt == VEC_F32) {
    if (cpt == 4)
      vec_batch_c<float, 4>(op, args, items, n_items, dots, smem, st);
    else if (cpt == 2)
      vec_batch_c<float, 2>(op, args, items, n_items, dots, smem, st);
    else
      vec_batch_c<float, 1>(op, args, items, n_items, dots, smem, st);
  } else {
    if (cpt == 2)
      vec_batch_c<double, 2>(op, args, items, n_items, dots, smem, st);
    else
      vec_batch_c<double, 1>(op, args, items, n_items, dots, smem, st);
  }
}

// ---------------------------------------------------------------------------
// Batched dense coarsest-level solve (FP64 arithmetic).  Item = a row range
// [first_slot, row_end) of one problem's coarsest level.
template <typename T>
__global__ void __launch_bounds__(kBlock) coarse_batch_kernel(const CoarseArgs* __restrict__ args,
                                                             const BItem* __restrict__ items, int32_t n_items) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const BItem bi = items[it];
    const CoarseArgs a = args[bi.arg];
    if (a.skip && *a.skip == 0) continue;
    const T* Y = static_cast<const T*>(a.Y);
    T* Z = static_cast<T*>(a.Z);
    const int64_t r0 = bi.first_slot, r1 = bi.row_end;
    const int64_t total = (r1 - r0) * a.C;
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      const int64_t i = r0 + t / a.C, c = t % a.C;
      const double* row = a.Ainv + i * a.n;
      double acc0 = 0.0, acc1 = 0.0;
      int j = 0;
      for (; j + 1 < a.n; j += 2) {
        acc0 = fma(row[j], (double)Y[(int64_t)j * a.C + c], acc0);
        acc1 = fma(row[j + 1], (double)Y[(int64_t)(j + 1) * a.C + c], acc1);
      }
      if (j < a.n) acc0 = fma(row[j], (double)Y[(int64_t)j * a.C + c], acc0);
      Z[i * a.C + c] = (T)(acc0 + acc1);
    }
  }
}

void launch_coarse_batch(VecType vt, const CoarseArgs* args, const BItem* items, int32_t n_items, cudaStream_t st) {
  if (n_items <= 0) return;
  count_launch();
  const int g = std::min<int>(n_items, max_grid_blocks());
  if (vt == VEC_F64)
    coarse_batch_kernel<double><<<g, kBlock, 0, st>>>(args, items, n_items);
  else
    coarse_batch_kernel<float><<<g, kBlock, 0, st>>>(args, items, n_items);
}

}  // namespace amgsym
