// Symmetry transforms, PCG vector updates, the dense coarsest-level solve and
// the adjoint coefficient gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "coarse.cuh"
#include "device.h"
#include "dot.cuh"

namespace amgsym {

static int g_sms = 0;
static std::atomic<int64_t> g_launches{0};

void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int num_sms() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

// Grid-stride kernels run at most 8 resident 256-thread blocks per SM (2048 threads).
int max_grid_blocks() { return num_sms() * 8; }

int resident_grid(const void* kernel, size_t smem_bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(kernel, smem_bytes);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem_bytes) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();  // not cached: fall back to the static bound this time
    return max_grid_blocks();
  }
  const int g = num_sms() * std::min(per_sm, 8);
  cache[key] = g;
  return g;
}

static int grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, max_grid_blocks()));
}

// ---------------------------------------------------------------------------
// Forward transform (Alg. 1, "Transform forward"; eq. "P_s" without the
// 2^{-s/2} factor): gather the 2^s mirror images of every base cell through
// perm, then s butterfly stages (a + b, a - b).  One thread per (rhs, l);
// consecutive threads take consecutive l so the gathers of each copy and the
// interleaved writes are coalesced.

template <int S, typename OT>
__global__ void __launch_bounds__(kBlock) transform_fwd_kernel(const double* __restrict__ b, int32_t nrhs,
                                                               int64_t ld, const int32_t* __restrict__ perm,
                                                               int64_t n_b, OT* __restrict__ xhat) {
  constexpr int NB = 1 << S;
  const int64_t total = n_b * nrhs;
  const int64_t C = (int64_t)nrhs * NB;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n_b, l = t - r * n_b;
    double v[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) v[j] = __ldcs(b + r * ld + __ldcs(perm + j * n_b + l));
#pragma unroll
    for (int st = 0; st < S; ++st) {
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (!(i & (1 << st))) {
          const double a0 = v[i], a1 = v[i | (1 << st)];
          v[i] = a0 + a1;
          v[i | (1 << st)] = a0 - a1;
        }
    }
    OT* o = xhat + l * C + r * NB;
#pragma unroll
    for (int i = 0; i < NB; ++i) o[i] = (OT)v[i];
  }
}

template <int S, typename IT>
__global__ void __launch_bounds__(kBlock) transform_bwd_kernel(const IT* __restrict__ xhat, int32_t nrhs,
                                                               const int32_t* __restrict__ perm, int64_t n_b,
                                                               double* __restrict__ x, int64_t ld) {
  constexpr int NB = 1 << S;
  const int64_t total = n_b * nrhs;
  const int64_t C = (int64_t)nrhs * NB;
  const double scale = 1.0 / (double)NB;  // 2^{-s}: exact
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n_b, l = t - r * n_b;
    double v[NB];
    const IT* in = xhat + l * C + r * NB;
#pragma unroll
    for (int i = 0; i < NB; ++i) v[i] = (double)in[i];
#pragma unroll
    for (int st = 0; st < S; ++st) {
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (!(i & (1 << st))) {
          const double a0 = v[i], a1 = v[i | (1 << st)];
          v[i] = a0 + a1;
          v[i | (1 << st)] = a0 - a1;
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) __stcs(x + r * ld + __ldcs(perm + j * n_b + l), v[j] * scale);
  }
}

template <typename OT>
static void fwd_dispatch(const double* b, int32_t nrhs, int64_t ld, const int32_t* perm, int64_t n_b, int32_t s,
                         OT* xhat, cudaStream_t st) {
  const int g = grid_for(n_b * nrhs, kBlock);
  switch (s) {
    case 0: transform_fwd_kernel<0, OT><<<g, kBlock, 0, st>>>(b, nrhs, ld, perm, n_b, xhat); break;
    case 1: transform_fwd_kernel<1, OT><<<g, kBlock, 0, st>>>(b, nrhs, ld, perm, n_b, xhat); break;
    case 2: transform_fwd_kernel<2, OT><<<g, kBlock, 0, st>>>(b, nrhs, ld, perm, n_b, xhat); break;
    case 3: transform_fwd_kernel<3, OT><<<g, kBlock, 0, st>>>(b, nrhs, ld, perm, n_b, xhat); break;
    case 4: transform_fwd_kernel<4, OT><<<g, kBlock, 0, st>>>(b, nrhs, ld, perm, n_b, xhat); break;
    default: fail(AMGSYM_ERR_ARG, "the device transform supports s <= 4");
  }
}

void launch_transform_fwd(const double* b, int32_t nrhs, int64_t ld, const int32_t* perm, int64_t n_b, int32_t s,
                          void* xhat, VecType ot, cudaStream_t st) {
  count_launch();
  if (ot == VEC_F64)
    fwd_dispatch<double>(b, nrhs, ld, perm, n_b, s, static_cast<double*>(xhat), st);
  else
    fwd_dispatch<float>(b, nrhs, ld, perm, n_b, s, static_cast<float*>(xhat), st);
}

template <typename IT>
static void bwd_dispatch(const IT* xhat, int32_t nrhs, const int32_t* perm, int64_t n_b, int32_t s, double* x,
                         int64_t ld, cudaStream_t st) {
  const int g = grid_for(n_b * nrhs, kBlock);
  switch (s) {
    case 0: transform_bwd_kernel<0, IT><<<g, kBlock, 0, st>>>(xhat, nrhs, perm, n_b, x, ld); break;
    case 1: transform_bwd_kernel<1, IT><<<g, kBlock, 0, st>>>(xhat, nrhs, perm, n_b, x, ld); break;
    case 2: transform_bwd_kernel<2, IT><<<g, kBlock, 0, st>>>(xhat, nrhs, perm, n_b, x, ld); break;
    case 3: transform_bwd_kernel<3, IT><<<g, kBlock, 0, st>>>(xhat, nrhs, perm, n_b, x, ld); break;
    case 4: transform_bwd_kernel<4, IT><<<g, kBlock, 0, st>>>(xhat, nrhs, perm, n_b, x, ld); break;
    default: fail(AMGSYM_ERR_ARG, "the device transform supports s <= 4");
  }
}

void launch_transform_bwd(const void* xhat, VecType it, int32_t nrhs, const int32_t* perm, int64_t n_b, int32_t s,
                          double* x, int64_t ld, cudaStream_t st) {
  count_launch();
  if (it == VEC_F64)
    bwd_dispatch<double>(static_cast<const double*>(xhat), nrhs, perm, n_b, s, x, ld, st);
  else
    bwd_dispatch<float>(static_cast<const float*>(xhat), nrhs, perm, n_b, s, x, ld, st);
}

// ---------------------------------------------------------------------------
// PCG updates.  Element e of a [rows][C] array belongs to column e % C; the
// thread mapping is the SpMM's (thread owns CPT columns of a row slot) so the
// fused dot reduction is shared.

template <typename T, int N>
struct alignas(sizeof(T) * N) VecM {
  T v[N];
};

template <typename T>
struct DotAcc {
  using type = float;
};
template <>
struct DotAcc<double> {
  using type = double;
};

template <typename T, int CPT, bool HAS_DOT>
__global__ void __launch_bounds__(kBlock) cg_update1_kernel(int64_t rows, int32_t C, T* __restrict__ x,
                                                            T* __restrict__ r, const T* __restrict__ p,
                                                            const T* __restrict__ q, DotArgs dot,
                                                            const int32_t* skip) {
  using DT = typename DotAcc<T>::type;
  using V = VecM<T, CPT>;
  if (skip && *skip == 0) return;
  const int TPR = C / CPT;
  const int rows_pb = kBlock / TPR;
  const int rloc = threadIdx.x / TPR;
  const int c0 = (threadIdx.x % TPR) * CPT;
  const bool has_cols = rloc < rows_pb;
  T al[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) al[k] = (T)dot.sc.alpha[c0 + k];
  DT part[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) part[k] = (DT)0;
  if (has_cols) {
    for (int64_t row = blockIdx.x * (int64_t)rows_pb + rloc; row < rows; row += (int64_t)gridDim.x * rows_pb) {
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
  }
  if (HAS_DOT) {
    extern __shared__ double sm[];
    double pd[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) pd[k] = has_cols ? (double)part[k] : 0.0;
    block_dot<CPT>(dot, pd, c0, has_cols, rloc, rows_pb, TPR, C, sm, blockIdx.x, gridDim.x, dot.sc.partials,
                   dot.sc.ticket);
  }
}

template <typename T, int CPT>
static void update1_c(int64_t rows, int32_t C, void* x, void* r, const void* p, const void* q, const DotArgs& dot,
                      cudaStream_t st, const int32_t* skip) {
  const int rows_pb = kBlock / (C / CPT);
  const size_t smem = sizeof(double) * (size_t)dot_smem_doubles(C / CPT, rows_pb, C);
  int g = grid_for(rows, rows_pb > 0 ? rows_pb : 1);
  g = std::min(g, resident_grid((const void*)cg_update1_kernel<T, CPT, true>, smem));
  if ((int64_t)g * C > dot.sc.partial_cap) g = (int)(dot.sc.partial_cap / C);
  cg_update1_kernel<T, CPT, true><<<g, kBlock, smem, st>>>(rows, C, static_cast<T*>(x), static_cast<T*>(r),
                                                        static_cast<const T*>(p), static_cast<const T*>(q), dot, skip);
}

template <typename T>
static void update1_t(int64_t rows, int32_t C, void* x, void* r, const void* p, const void* q, const DotArgs& dot,
                      cudaStream_t st, const int32_t* skip) {
  constexpr int V = 16 / (int)sizeof(T);
  if (V >= 4 && C % 4 == 0)
    update1_c<T, (V >= 4 ? 4 : 1)>(rows, C, x, r, p, q, dot, st, skip);
  else if (C % 2 == 0)
    update1_c<T, 2>(rows, C, x, r, p, q, dot, st, skip);
  else
    update1_c<T, 1>(rows, C, x, r, p, q, dot, st, skip);
}

void launch_cg_update1(VecType vt, int64_t rows, int32_t C, void* x, void* r, const void* p, const void* q,
                       const DotArgs& dot, cudaStream_t st, const int32_t* skip) {
  count_launch();
  if (vt == VEC_F64)
    update1_t<double>(rows, C, x, r, p, q, dot, st, skip);
  else
    update1_t<float>(rows, C, x, r, p, q, dot, st, skip);
}

// p = z + beta p, CPT columns per thread with vector loads.
template <typename T, int CPT>
__global__ void __launch_bounds__(kBlock) cg_update2_kernel(int64_t rows, int32_t C, T* __restrict__ p,
                                                            const T* __restrict__ z, const double* __restrict__ beta,
                                                            const int32_t* skip) {
  using V = VecM<T, CPT>;
  if (skip && *skip == 0) return;
  const int TPR = C / CPT;
  const int rows_pb = kBlock / TPR;
  const int rloc = threadIdx.x / TPR;
  const int c0 = (threadIdx.x % TPR) * CPT;
  if (rloc >= rows_pb) return;
  T b[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) b[k] = (T)beta[c0 + k];
  for (int64_t row = blockIdx.x * (int64_t)rows_pb + rloc; row < rows; row += (int64_t)gridDim.x * rows_pb) {
    const int64_t o = row * C + c0;
    V pv = *reinterpret_cast<const V*>(p + o);
    const V zv = *reinterpret_cast<const V*>(z + o);
#pragma unroll
    for (int k = 0; k < CPT; ++k) pv.v[k] = zv.v[k] + b[k] * pv.v[k];
    *reinterpret_cast<V*>(p + o) = pv;
  }
}

template <typename T, int CPT>
static void update2_c(int64_t rows, int32_t C, void* p, const void* z, const double* beta, cudaStream_t st,
                      const int32_t* skip) {
  const int rows_pb = kBlock / (C / CPT);
  const int g = grid_for(rows, rows_pb > 0 ? rows_pb : 1);
  cg_update2_kernel<T, CPT><<<g, kBlock, 0, st>>>(rows, C, static_cast<T*>(p), static_cast<const T*>(z), beta, skip);
}

template <typename T>
static void update2_t(int64_t rows, int32_t C, void* p, const void* z, const double* beta, cudaStream_t st,
                      const int32_t* skip) {
  constexpr int V = 16 / (int)sizeof(T);
  if (V >= 4 && C % 4 == 0)
    update2_c<T, (V >= 4 ? 4 : 1)>(rows, C, p, z, beta, st, skip);
  else if (C % 2 == 0)
    update2_c<T, 2>(rows, C, p, z, beta, st, skip);
  else
    update2_c<T, 1>(rows, C, p, z, beta, st, skip);
}

void launch_cg_update2(VecType vt, int64_t rows, int32_t C, void* p, const void* z, const double* beta,
                       cudaStream_t st, const int32_t* skip) {
  count_launch();
  if (vt == VEC_F64)
    update2_t<double>(rows, C, p, z, beta, st, skip);
  else
    update2_t<float>(rows, C, p, z, beta, st, skip);
}

// Diagonal smoother step (a diagonal FSAI factor: omega G^T G = diag(jd)).
// One thread per row slice of V columns: z = jd[row] * src (or + z, fused).
template <typename T, int V>
__global__ void __launch_bounds__(kBlock) jacobi_kernel(int64_t rows, int32_t C, const T* __restrict__ jd,
                                                        const T* __restrict__ src, T* z, int accumulate,
                                                        const int32_t* skip) {
  if (skip && *skip == 0) return;
  const int64_t slices = (int64_t)rows * (C / V);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < slices; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / (C / V);
    const T d = jd[row];
    const int64_t e = t * V;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const T s = src[e + q];
      z[e + q] = accumulate ? fma(d, s, z[e + q]) : d * s;
    }
  }
}

void launch_jacobi(VecType vt, int64_t rows, int32_t C, const void* jd, const void* src, void* z, int accumulate,
                   cudaStream_t st, const int32_t* skip) {
  count_launch();
  if (vt == VEC_F64) {
    const double* j = static_cast<const double*>(jd);
    const double* s = static_cast<const double*>(src);
    double* d = static_cast<double*>(z);
    if (C % 2 == 0)
      jacobi_kernel<double, 2><<<grid_for(rows * (C / 2), kBlock), kBlock, 0, st>>>(rows, C, j, s, d, accumulate, skip);
    else
      jacobi_kernel<double, 1><<<grid_for(rows * C, kBlock), kBlock, 0, st>>>(rows, C, j, s, d, accumulate, skip);
  } else {
    const float* j = static_cast<const float*>(jd);
    const float* s = static_cast<const float*>(src);
    float* d = static_cast<float*>(z);
    if (C % 4 == 0)
      jacobi_kernel<float, 4><<<grid_for(rows * (C / 4), kBlock), kBlock, 0, st>>>(rows, C, j, s, d, accumulate, skip);
    else
      jacobi_kernel<float, 1><<<grid_for(rows * C, kBlock), kBlock, 0, st>>>(rows, C, j, s, d, accumulate, skip);
  }
}

template <typename T>
__global__ void add_to_f64_kernel(int64_t count, double* __restrict__ y, const T* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    y[e] += (double)x[e];
}

void launch_add_to_f64(VecType xt, int64_t count, double* y, const void* x, cudaStream_t st) {
  count_launch();
  const int g = grid_for(count, kBlock);
  if (xt == VEC_F64)
    add_to_f64_kernel<double><<<g, kBlock, 0, st>>>(count, y, static_cast<const double*>(x));
  else
    add_to_f64_kernel<float><<<g, kBlock, 0, st>>>(count, y, static_cast<const float*>(x));
}

template <typename T>
__global__ void copy_kernel(int64_t count, T* __restrict__ d, const T* __restrict__ s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = s[e];
}

void launch_copy(VecType vt, int64_t count, void* dst, const void* src, cudaStream_t st) {
  count_launch();
  const int g = grid_for(count, kBlock);
  if (vt == VEC_F64)
    copy_kernel<double><<<g, kBlock, 0, st>>>(count, static_cast<double*>(dst), static_cast<const double*>(src));
  else
    copy_kernel<float><<<g, kBlock, 0, st>>>(count, static_cast<float*>(dst), static_cast<const float*>(src));
}

template <typename T>
__global__ void zero_kernel(int64_t count, T* __restrict__ d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (T)0;
}

void launch_zero(VecType vt, int64_t count, void* dst, cudaStream_t st) {
  count_launch();
  const int g = grid_for(count, kBlock);
  if (vt == VEC_F64)
    zero_kernel<double><<<g, kBlock, 0, st>>>(count, static_cast<double*>(dst));
  else
    zero_kernel<float><<<g, kBlock, 0, st>>>(count, static_cast<float*>(dst));
}

// Per-column dots of two [rows][C] vectors.  A thread owns CPT consecutive
// columns (one 16-byte vector where C allows) of its row slots and sums their
// products in the vector precision (DotAcc: FP32 for FP32 vectors, as the
// fused dots of the SpMM epilogues; the FP64 rate of this GPU is a small
// fraction of its FP32 rate), then the block and grid combine the per-thread
// partials in FP64 in a fixed order.
template <typename T, int CPT>
__global__ void __launch_bounds__(kBlock) dot_kernel(int64_t rows, int32_t C, const T* __restrict__ a,
                                                     const T* __restrict__ b, DotArgs dot, const int32_t* skip) {
  using DT = typename DotAcc<T>::type;
  using V = VecM<T, CPT>;
  if (skip && *skip == 0) return;
  const int TPR = C / CPT;
  const int rows_pb = kBlock / TPR;
  const int rloc = threadIdx.x / TPR;
  const int c0 = (threadIdx.x % TPR) * CPT;
  const bool has_cols = rloc < rows_pb;
  DT acc[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) acc[k] = (DT)0;
  if (has_cols)
    for (int64_t row = blockIdx.x * (int64_t)rows_pb + rloc; row < rows; row += (int64_t)gridDim.x * rows_pb) {
      const V av = *reinterpret_cast<const V*>(a + row * C + c0);
      const V bv = *reinterpret_cast<const V*>(b + row * C + c0);
#pragma unroll
      for (int k = 0; k < CPT; ++k) acc[k] = fma((DT)av.v[k], (DT)bv.v[k], acc[k]);
    }
  double part[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) part[k] = has_cols ? (double)acc[k] : 0.0;
  extern __shared__ double sm[];
  block_dot<CPT>(dot, part, c0, has_cols, rloc, rows_pb, TPR, C, sm, blockIdx.x, gridDim.x, dot.sc.partials,
                 dot.sc.ticket);
}

template <typename T, int CPT>
static void dot_c(int64_t rows, int32_t C, const void* a, const void* b, const DotArgs& dot, cudaStream_t st,
                  const int32_t* skip) {
  const int TPR = C / CPT, rows_pb = kBlock / TPR;
  int g = grid_for(rows, rows_pb > 0 ? rows_pb : 1);
  if ((int64_t)g * C > dot.sc.partial_cap) g = (int)(dot.sc.partial_cap / C);
  const size_t smem = sizeof(double) * (size_t)dot_smem_doubles(TPR, rows_pb, C);
  dot_kernel<T, CPT><<<g, kBlock, smem, st>>>(rows, C, static_cast<const T*>(a), static_cast<const T*>(b), dot, skip);
}

void launch_dot(VecType vt, int64_t rows, int32_t C, const void* a, const void* b, const DotArgs& dot,
                cudaStream_t st, const int32_t* skip) {
  count_launch();
  if (vt == VEC_F64) {
    if (C % 2 == 0)
      dot_c<double, 2>(rows, C, a, b, dot, st, skip);
    else
      dot_c<double, 1>(rows, C, a, b, dot, st, skip);
  } else {
    if (C % 4 == 0)
      dot_c<float, 4>(rows, C, a, b, dot, st, skip);
    else if (C % 2 == 0)
      dot_c<float, 2>(rows, C, a, b, dot, st, skip);
    else
      dot_c<float, 1>(rows, C, a, b, dot, st, skip);
  }
}

// ---------------------------------------------------------------------------
// Coarsest level (Sec. 5: "a direct method solves the coarsest level"):
// Z = A_c^{-1} Y with the precomputed FP64 inverse; FP64 arithmetic, one warp
// per row (coarse.cuh).
template <typename T>
__global__ void __launch_bounds__(kBlock) coarse_kernel(int32_t n, int32_t C, const double* __restrict__ Ainv,
                                                        const T* __restrict__ Y, T* __restrict__ Z,
                                                        const int32_t* skip) {
  if (skip && *skip == 0) return;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  coarse_rows_warp<T>(n, C, Ainv, Y, Z, warp, nwarps, [](const T* p) { return __ldg(p); });
}

void launch_coarse_solve(VecType vt, int32_t n, int32_t C, const double* Ainv, const void* Y, void* Z,
                         cudaStream_t st, const int32_t* skip) {
  count_launch();
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 7) / 8, max_grid_blocks()));
  if (vt == VEC_F64)
    coarse_kernel<double><<<g, kBlock, 0, st>>>(n, C, Ainv, static_cast<const double*>(Y), static_cast<double*>(Z), skip);
  else
    coarse_kernel<float><<<g, kBlock, 0, st>>>(n, C, Ainv, static_cast<const float*>(Y), static_cast<float*>(Z), skip);
}

// ---------------------------------------------------------------------------
// Singular (pure Neumann) problems: the constant vector spans the null space.
// In the reduced layout the full-grid constant is block 0 of every RHS (the
// all-"+" combination), so removing the constant component of a natural-order
// vector is removing the mean of its columns r*nb, r = 0..nrhs-1.
// Deterministic: per-block partial sums in a fixed tree, one block adds the
// partials in block order, then the subtraction.
__global__ void __launch_bounds__(kBlock) block0_partial_kernel(const double* __restrict__ X, int64_t rows,
                                                                int32_t C, int32_t nb, int32_t nrhs,
                                                                double* __restrict__ part) {
  __shared__ double sm[kBlock];
  for (int32_t r = 0; r < nrhs; ++r) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < rows; i += (int64_t)gridDim.x * kBlock)
      acc += X[i * C + (int64_t)r * nb];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kBlock / 2; w >= 1; w >>= 1) {
      if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * nrhs + r] = sm[0];
    __syncthreads();
  }
}

__global__ void block0_mean_kernel(double* part, int32_t nblocks, int32_t nrhs, int64_t rows) {
  for (int32_t r = threadIdx.x; r < nrhs; r += blockDim.x) {
    double acc = 0.0;
    for (int32_t g = 0; g < nblocks; ++g) acc += part[(int64_t)g * nrhs + r];
    part[(int64_t)nblocks * nrhs + r] = acc / (double)rows;
  }
}

__global__ void __launch_bounds__(kBlock) block0_sub_kernel(double* __restrict__ X, int64_t rows, int32_t C,
                                                            int32_t nb, int32_t nrhs, const double* __restrict__ mean) {
  const int64_t total = rows * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x; t < total; t += (int64_t)gridDim.x * kBlock) {
    const int64_t i = t / nrhs;
    const int32_t r = (int32_t)(t - i * nrhs);
    X[i * C + (int64_t)r * nb] -= mean[r];
  }
}

void launch_sub_block0_mean(double* X, int64_t rows, int32_t nrhs, int32_t nb, double* scratch,
                            int64_t scratch_cap, cudaStream_t st) {
  const int32_t C = nrhs * nb;
  int64_t g = std::min<int64_t>(max_grid_blocks(), (rows + kBlock - 1) / kBlock);
  g = std::max<int64_t>(1, std::min<int64_t>(g, scratch_cap / nrhs - 1));
  count_launch(3);
  block0_partial_kernel<<<(int)g, kBlock, 0, st>>>(X, rows, C, nb, nrhs, scratch);
  block0_mean_kernel<<<1, 256, 0, st>>>(scratch, (int32_t)g, nrhs, rows);
  block0_sub_kernel<<<grid_for(rows * nrhs, kBlock), kBlock, 0, st>>>(X, rows, C, nb, nrhs, scratch + g * nrhs);
}

// ---------------------------------------------------------------------------
// AMGR coarse step: between the transformed layout of Alg. 1 ([n_cb][nrhs *
// 2^s], column r * 2^s + i = block i) and the full coarse domain of the
// coarse problem ([n_cb * 2^s][nrhs], row l * 2^s + j = copy j), by the
// Walsh-Hadamard butterfly of eq. "P_s": out_j = scale * sum_i s(i, j) in_i
// with s(i, j) = (-1)^popcount(i & j) (dir 0: scale 2^-s; dir 1: scale 1),
// as the fast transform (log2(nb) stages of sums and differences) in the
// vector precision.  dir 0 may also take an epilogue: out = alpha * (the
// butterfly) + beta * Z (Z in the output layout; beta = 0 reads no Z),
// e.g. the residual y - A_c z.
template <typename T, int NB>
__global__ void __launch_bounds__(kBlock) coarse_relayout_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                 int64_t ncb, int32_t nrhs, int dir, double alpha,
                                                                 double beta, const T* __restrict__ Z) {
  const int64_t total = ncb * nrhs;
  const T scale = dir == 0 ? (T)(alpha / NB) : (T)1;
  const T tb = (T)beta;
  for (int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x; t < total; t += (int64_t)gridDim.x * kBlock) {
    const int64_t l = t / nrhs;
    const int32_t r = (int32_t)(t - l * nrhs);
    T v[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      v[i] = dir == 0 ? in[l * nrhs * NB + (int64_t)r * NB + i] : in[(l * NB + i) * nrhs + r];
#pragma unroll
    for (int h = 1; h < NB; h <<= 1)
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (!(i & h)) {
          const T a = v[i], b = v[i + h];
          v[i] = a + b;
          v[i + h] = a - b;
        }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (dir == 0) {
        const int64_t o = (l * NB + j) * nrhs + r;
        out[o] = beta != 0.0 ? scale * v[j] + tb * Z[o] : scale * v[j];
      } else {
        out[l * nrhs * NB + (int64_t)r * NB + j] = v[j];
      }
    }
  }
}

template <typename T>
static void relayout_t(const void* in, void* out, int64_t ncb, int32_t nrhs, int32_t nb, int dir, double alpha,
                       double beta, const void* Z, int g, cudaStream_t st) {
  const T* i = static_cast<const T*>(in);
  T* o = static_cast<T*>(out);
  const T* z = static_cast<const T*>(Z);
  switch (nb) {
    case 1: coarse_relayout_kernel<T, 1><<<g, kBlock, 0, st>>>(i, o, ncb, nrhs, dir, alpha, beta, z); break;
    case 2: coarse_relayout_kernel<T, 2><<<g, kBlock, 0, st>>>(i, o, ncb, nrhs, dir, alpha, beta, z); break;
    case 4: coarse_relayout_kernel<T, 4><<<g, kBlock, 0, st>>>(i, o, ncb, nrhs, dir, alpha, beta, z); break;
    case 8: coarse_relayout_kernel<T, 8><<<g, kBlock, 0, st>>>(i, o, ncb, nrhs, dir, alpha, beta, z); break;
    case 16: coarse_relayout_kernel<T, 16><<<g, kBlock, 0, st>>>(i, o, ncb, nrhs, dir, alpha, beta, z); break;
    default: fail(AMGSYM_ERR_ARG, "coarse relayout: 2^s must be at most 16");
  }
}

void launch_coarse_relayout(VecType vt, const void* in, void* out, int64_t ncb, int32_t nrhs, int32_t nb, int dir,
                            cudaStream_t st, double alpha, double beta, const void* Z) {
  count_launch();
  const int g = grid_for(ncb * nrhs, kBlock);
  if (vt == VEC_F64)
    relayout_t<double>(in, out, ncb, nrhs, nb, dir, alpha, beta, Z, g, st);
  else
    relayout_t<float>(in, out, ncb, nrhs, nb, dir, alpha, beta, Z, g, st);
}

__global__ void hold_kernel(int32_t naps) {
  for (int32_t i = 0; i < naps; ++i) __nanosleep(10000);
}

void launch_hold(int32_t naps, cudaStream_t st) {
  count_launch();
  hold_kernel<<<1, 1, 0, st>>>(std::max<int32_t>(0, std::min<int32_t>(naps, 2000)));
}

__global__ void set_value_kernel(double* dst, double v) { *dst = v; }

void launch_set_value(double* dst, double v, cudaStream_t st) {
  count_launch();
  set_value_kernel<<<1, 1, 0, st>>>(dst, v);
}

__global__ void init_scalars_kernel(DevScalars sc, int32_t nrhs, int32_t nb) {
  __shared__ int n_act;
  if (threadIdx.x == 0) n_act = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < nrhs * nb; c += blockDim.x) {
    const int r = c / nb;
    const int act = sc.bnorm2[r] > 0.0 ? 1 : 0;
    sc.active[c] = act;
    sc.alpha[c] = 0.0;
    sc.beta[c] = 0.0;
    sc.rz[c] = 0.0;
    sc.rr[c] = 0.0;
    if (act && (c % nb) == 0) atomicAdd(&n_act, 1);
  }
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) sc.relres[r] = sc.bnorm2[r] > 0.0 ? 1.0 : 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    sc.status[0] = n_act;
    sc.status[1] = 0;
    sc.status[2] = 0;
    *sc.ticket = 0u;
  }
}

void launch_init_scalars(const DevScalars& sc, int32_t nrhs, int32_t nb, cudaStream_t st) {
  count_launch();
  init_scalars_kernel<<<1, kBlock, 0, st>>>(sc, nrhs, nb);
}

// ---------------------------------------------------------------------------
// Adjoint coefficient gradient (see amgsym_fv_grad_logk): one thread per cell,
// both faces of every axis, FP64.
struct GridDev {
  int32_t d;
  int64_t N[3];
  int64_t off[3];
};

__global__ void __launch_bounds__(kBlock) fv_grad_kernel(GridDev g, const double* __restrict__ w,
                                                         const double* __restrict__ k, const double* __restrict__ u,
                                                         const double* __restrict__ lam, int32_t nrhs, int64_t ld,
                                                         double* __restrict__ grad, int32_t accumulate) {
  const int64_t n = g.N[0] * g.N[1] * g.N[2];
  const int64_t stride[3] = {1, g.N[0], g.N[0] * g.N[1]};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t c[3];
    c[0] = p % g.N[0];
    c[1] = (p / g.N[0]) % g.N[1];
    c[2] = p / (g.N[0] * g.N[1]);
    const double kp = k[p];
    double acc = 0.0;
    for (int a = 0; a < g.d; ++a) {
      double area = 1.0;
      for (int b = 0; b < g.d; ++b)
        if (b != a) area *= w[g.off[b] + c[b]];
      const double hp = w[g.off[a] + c[a]];
      const double rp = hp / (2.0 * kp);
      const double dtdg_fac = hp / (2.0 * area * kp);  // dt/dg_p = t^2 * this
      for (int side = 0; side < 2; ++side) {
        const bool interior = side == 0 ? c[a] > 0 : c[a] < g.N[a] - 1;
        double t;
        int64_t q = -1;
        if (interior) {
          q = side == 0 ? p - stride[a] : p + stride[a];
          const double hq = w[g.off[a] + c[a] + (side == 0 ? -1 : 1)];
          t = area / (rp + hq / (2.0 * k[q]));
        } else {
          t = area / rp;
        }
        double dLdt = 0.0;
        for (int r = 0; r < nrhs; ++r) {
          const double up = u[r * ld + p], lp = lam[r * ld + p];
          if (interior)
            dLdt -= (lp - lam[r * ld + q]) * (up - u[r * ld + q]);
          else
            dLdt -= lp * up;
        }
        acc += dLdt * t * t * dtdg_fac;
      }
    }
    grad[p] = accumulate ? grad[p] + acc : acc;
  }
}

void launch_fv_grad(int32_t d, const int64_t* N, const double* widths, const double* k, const double* u,
                    const double* lam, int32_t nrhs, int64_t ld, double* grad, int32_t accumulate,
                    cudaStream_t st) {
  count_launch();
  GridDev g;
  g.d = d;
  int64_t off = 0;
  for (int a = 0; a < 3; ++a) {
    g.N[a] = a < d ? N[a] : 1;
    g.off[a] = off;
    if (a < d) off += N[a];
  }
  const int64_t n = g.N[0] * g.N[1] * g.N[2];
  fv_grad_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(g, widths, k, u, lam, nrhs, ld, grad, accumulate);
}

}  // namespace amgsym
