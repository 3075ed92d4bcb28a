// The coarse end of the V-cycle as one persistent kernel.
//
// Below some size the levels of the hierarchy (Alg. "apply" shape, Sec. 3.2)
// hold too few rows to fill the GPU, and one launch per product costs more
// than the product: a V-cycle over the coarsest levels is a chain of small
// dependent SpMMs (smoother, residual, restriction, prolongation) and the
// dense coarsest solve.  Here that chain runs as the phases of one
// cooperative kernel: every block takes the rows of a phase grid-stride with
// the same tile code as the stand-alone kernels (so the products and their
// summation order are the same), then waits at a grid barrier for the phase
// to finish everywhere.
//
// The barrier is a counter plus a generation word.  Every wait is bounded: a
// block that polls more than CycleBar::spins times (4 M polls with a 32 ns
// back-off by default, well above a second) sets the error word and
// returns, the other blocks then time out at the same or the next barrier,
// and the host reports the error.  The cooperative launch makes every block
// co-resident, so the bound is never reached in a correct run;
// amgsym_cycle_timeout_check makes it run out on purpose (a barrier that
// awaits one arrival more than the grid has, with a short bound).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "coarse.cuh"
#include "spmm_common.cuh"

namespace amgsym {

__device__ __forceinline__ bool grid_barrier(const CycleBar& b) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = b.gen;
    const unsigned g0 = *vgen;  // generation before arriving
    __threadfence();            // this block's writes before the arrival
    if (atomicAdd(b.count, 1u) + 1u == gridDim.x + b.extra) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);  // release every waiter
    } else {
      // poll with plain (volatile, L2) loads: no atomic traffic on the line
      // the arrivals update
      long long it = 0;
      while (*vgen == g0) {
        if (++it > b.spins) {
          atomicExch(b.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();  // the other blocks' writes before this block's reads
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Dense coarsest solve Z = Ainv Y in FP64 arithmetic, the warp-per-row order
// of the stand-alone coarse kernel (coarse.cuh).
template <typename XT>
__device__ __forceinline__ void dense_phase(const CoarseArgs& c) {
  // Y was written earlier in the launch: L2 loads
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  coarse_rows_warp<XT>(c.n, c.C, c.Ainv, static_cast<const XT*>(c.Y), static_cast<XT*>(c.Z), warp, nwarps,
                       [](const XT* p) { return ldv_cg<XT, 1>(p).v[0]; });
}

// Diagonal smoother step, the arithmetic of the stand-alone jacobi kernel.
template <typename XT>
__device__ __forceinline__ void jacobi_phase(const JacobiArgs& j) {
  const int64_t total = j.rows * j.C;
  const XT* __restrict__ jd = static_cast<const XT*>(j.jd);
  const XT* src = static_cast<const XT*>(j.src);  // written earlier in the launch: L2 loads
  XT* z = static_cast<XT*>(j.z);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const XT d = __ldg(jd + e / j.C);
    const XT sv = ldv_cg<XT, 1>(src + e).v[0];
    z[e] = j.accumulate ? fma(d, sv, ldv_cg<XT, 1>(z + e).v[0]) : d * sv;
  }
}

template <typename MT, typename XT, int CPT>
__global__ void __launch_bounds__(kBlock, 2)
    cycle_kernel(const CyclePhase* __restrict__ phases, int32_t nphases, CycleBar bar, const int32_t* skip) {
  using DT = typename AccOf<XT>::type;
  __shared__ __align__(16) unsigned char raw[sizeof(CyclePhase)];
  CyclePhase& ph = *reinterpret_cast<CyclePhase*>(raw);
  if (skip && *skip == 0) return;  // uniform over the grid
  static_assert(sizeof(CyclePhase) % 4 == 0, "phase record in 4-byte words");
  constexpr int kWords = (int)(sizeof(CyclePhase) / 4);
  for (int k = 0; k < nphases; ++k) {
    __syncthreads();  // the previous phase is done with the record
    // the record in one round trip: a word per thread (read-only data)
    for (int w = threadIdx.x; w < kWords; w += blockDim.x)
      reinterpret_cast<unsigned*>(raw)[w] = __ldg(reinterpret_cast<const unsigned*>(phases + k) + w);
    __syncthreads();
    if (ph.kind == CYCLE_DENSE) {
      dense_phase<XT>(ph.c);
    } else if (ph.kind == CYCLE_JACOBI) {
      jacobi_phase<XT>(ph.j);
    } else {
      DT dpart[CPT];
      const SpmmArgs& a = ph.a;
      if (a.ndiag > 0) {
        spmm_tile<MT, XT, XT, CPT, 1, false, false, true, true>(a, blockIdx.x, gridDim.x, a.rows, dpart);
      } else {
        switch (a.kl) {
          case 1: spmm_tile<MT, XT, XT, CPT, 1, false, false, false, true>(a, blockIdx.x, gridDim.x, a.rows, dpart); break;
          case 2: spmm_tile<MT, XT, XT, CPT, 2, false, false, false, true>(a, blockIdx.x, gridDim.x, a.rows, dpart); break;
          case 4: spmm_tile<MT, XT, XT, CPT, 4, false, false, false, true>(a, blockIdx.x, gridDim.x, a.rows, dpart); break;
          case 8: spmm_tile<MT, XT, XT, CPT, 8, false, false, false, true>(a, blockIdx.x, gridDim.x, a.rows, dpart); break;
          default: spmm_tile<MT, XT, XT, CPT, 16, false, false, false, true>(a, blockIdx.x, gridDim.x, a.rows, dpart); break;
        }
      }
    }
    if (k + 1 < nphases && !grid_barrier(bar)) return;
  }
}

template <typename MT, typename XT, int CPT>
static const void* cycle_fn() {
  return (const void*)cycle_kernel<MT, XT, CPT>;
}

static const void* pick(ValType mt, VecType vt, int cpt) {
  if (mt == VAL_F32 && vt == VEC_F32) {
    switch (cpt) {
      case 8: return cycle_fn<float, float, 8>();
      case 4: return cycle_fn<float, float, 4>();
      case 2: return cycle_fn<float, float, 2>();
      default: return cycle_fn<float, float, 1>();
    }
  }
  if (mt == VAL_BF16 && vt == VEC_F32) {
    switch (cpt) {
      case 8: return cycle_fn<__nv_bfloat16, float, 8>();
      case 4: return cycle_fn<__nv_bfloat16, float, 4>();
      case 2: return cycle_fn<__nv_bfloat16, float, 2>();
      default: return cycle_fn<__nv_bfloat16, float, 1>();
    }
  }
  if (mt == VAL_F64 && vt == VEC_F64) {
    switch (cpt) {
      case 4: return cycle_fn<double, double, 4>();
      case 2: return cycle_fn<double, double, 2>();
      default: return cycle_fn<double, double, 1>();
    }
  }
  return nullptr;
}

int cycle_cpt(VecType vt, int32_t C) {
  const int V = vt == VEC_F64 ? 2 : 4;
  if (C % (2 * V) == 0) return 2 * V;
  if (C % V == 0) return V;
  if (C % 2 == 0) return 2;
  return 1;
}

int cycle_grid(ValType mt, VecType vt, int32_t C) {
  const void* fn = pick(mt, vt, cycle_cpt(vt, C));
  if (!fn) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0) != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  (void)per_sm;
  return num_sms();  // one block per SM: the fewest arrivals per barrier
}

cudaError_t launch_cycle(ValType mt, VecType vt, int32_t C, int grid, const CyclePhase* phases, int32_t nphases,
                         const CycleBar& bar, const int32_t* skip, cudaStream_t st) {
  const void* fn = pick(mt, vt, cycle_cpt(vt, C));
  if (!fn || grid < 1) return cudaErrorInvalidValue;
  count_launch();
  void* args[] = {(void*)&phases, (void*)&nphases, (void*)&bar, (void*)&skip};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace amgsym
