// Deterministic per-column dot products fused into kernel epilogues.
//
// Every participating kernel uses 256-thread blocks in which thread t owns
// the CPT consecutive columns c0 = (t % TPR) * CPT of row slot t / TPR.  A
// block reduces its threads' partials in shared memory in a fixed order,
// writes one partial per column to global memory, and the last block to
// finish (integer ticket) sums the block partials in a fixed order and runs
// the finalisation (CG scalars, convergence test).  No floating-point
// atomics: results are bit-reproducible run to run.
#pragma once

#include "device.h"

namespace amgsym {

constexpr int kBlock = 256;

__device__ __forceinline__ void dot_finalize_column(const DotArgs& d, int c, double sum) {
  DevScalars s = d.sc;
  switch (d.final) {
    case FIN_STORE_RZ:
      s.rz[c] = sum;
      break;
    case FIN_ALPHA: {
      const double rz = s.rz[c];
      double a = 0.0;
      if (s.active[c] && rz != 0.0) {
        if (sum > 0.0 && isfinite(sum)) a = rz / sum;
        else s.status[1] = 1;  // breakdown: p^T A p <= 0 or NaN
      }
      s.alpha[c] = a;
      break;
    }
    case FIN_BETA: {
      const double rz = s.rz[c];
      s.beta[c] = (s.active[c] && rz != 0.0) ? sum / rz : 0.0;
      s.rz[c] = sum;
      break;
    }
    case FIN_CONV:
      s.rr[c] = sum;
      break;
    default:
      break;
  }
}

// Per-RHS stage of FIN_CONV / FIN_STORE_BN; colsum in shared memory [C].
__device__ __forceinline__ void dot_finalize_rhs(const DotArgs& d, const double* colsum) {
  DevScalars s = d.sc;
  const int nrhs = d.cp.nrhs, nb = d.cp.nb;
  if (d.final == FIN_STORE_BN) {
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
      double t = 0.0;
      for (int i = 0; i < nb; ++i) t += colsum[r * nb + i];
      s.bnorm2[r] = t;
    }
    return;
  }
  if (d.final != FIN_CONV) return;
  __shared__ int n_active;
  if (threadIdx.x == 0) n_active = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += colsum[r * nb + i];
    const double bn = s.bnorm2[r];
    const double rel2 = bn > 0.0 ? t / bn : 0.0;
    s.relres[r] = sqrt(rel2);
    bool act = s.active[r * nb] != 0;
    if (act && !(rel2 > *s.tol2)) {  // converged (NaN keeps it active)
      act = false;
      for (int i = 0; i < nb; ++i) s.active[r * nb + i] = 0;
    }
    if (act) atomicAdd(&n_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.status[0] = n_active;
    if (d.cp.count_iter) s.status[2] += 1;
  }
}

// Block + grid reduction.  part[q] is this thread's partial for column
// c0 + q (zero when !has_cols).  Threads of one row slot are S consecutive
// lanes; when S is a power of two <= 32 the row slots of a warp are first
// combined with xor shuffles (lanes l, l^S, l^2S, ... share their columns),
// so shared memory holds one partial per warp and column; otherwise every
// slot gets its own line.  Shared scratch (dynamic): dot_smem_doubles(...).
// Every sum runs in a fixed assignment of threads to terms, so the order of
// additions, and the result, never varies from run to run.
__host__ __device__ inline int dot_smem_doubles(int S, int rows_pb, int C) {
  const bool pow2 = S > 0 && (S & (S - 1)) == 0 && S <= 32;
  const int lines = pow2 ? kBlock / 32 : rows_pb;
  return lines * C + kBlock + C;
}

template <int CPT>
__device__ __forceinline__ void block_dot(const DotArgs& d, double (&part)[CPT], int c0, bool has_cols,
                                          int rloc, int rows_pb, int S, int C, double* sm, int slot, int nslots,
                                          double* partials, unsigned* ticket) {
  const bool pow2 = (S & (S - 1)) == 0 && S <= 32;
  int lines;
  if (pow2) {
    for (int off = S; off < 32; off <<= 1) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) part[q] += __shfl_xor_sync(0xffffffffu, part[q], off);
    }
    lines = kBlock / 32;
    const int lane = threadIdx.x & 31;
    if (has_cols && lane < S) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) sm[(threadIdx.x >> 5) * C + c0 + q] = part[q];
    }
  } else {
    lines = rows_pb;
    if (has_cols) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) sm[rloc * C + c0 + q] = part[q];
    }
  }
  __syncthreads();
  const int slices = blockDim.x / C;  // C <= 256 = blockDim
  double* red = sm + lines * C;       // [slices][C], <= 256 doubles
  if ((int)threadIdx.x < slices * C) {
    const int c = threadIdx.x % C, sl = threadIdx.x / C;
    double t0 = 0.0, t1 = 0.0;
    int r = sl;
    for (; r + slices < lines; r += 2 * slices) {
      t0 += sm[r * C + c];
      t1 += sm[(r + slices) * C + c];
    }
    if (r < lines) t0 += sm[r * C + c];
    red[sl * C + c] = t0 + t1;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double t = 0.0;
    for (int sl = 0; sl < slices; ++sl) t += red[sl * C + c];
    partials[(int64_t)slot * C + c] = t;
  }
  __threadfence();
  __syncthreads();
  __shared__ unsigned is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == (unsigned)nslots - 1u) ? 1u : 0u;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if ((int)threadIdx.x < slices * C) {
    const int c = threadIdx.x % C, sl = threadIdx.x / C;
    const int nblk = nslots;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    int b = sl;
    for (; b + 3 * slices < nblk; b += 4 * slices) {
      t0 += __ldcg(partials + (int64_t)b * C + c);
      t1 += __ldcg(partials + (int64_t)(b + slices) * C + c);
      t2 += __ldcg(partials + (int64_t)(b + 2 * slices) * C + c);
      t3 += __ldcg(partials + (int64_t)(b + 3 * slices) * C + c);
    }
    for (; b < nblk; b += slices) t0 += __ldcg(partials + (int64_t)b * C + c);
    red[sl * C + c] = (t0 + t1) + (t2 + t3);
  }
  __syncthreads();
  double* colsum = sm;  // [C]
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double t = 0.0;
    for (int sl = 0; sl < slices; ++sl) t += red[sl * C + c];
    colsum[c] = t;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double t = colsum[c];
    if (d.coupled) {  // one CG per RHS: the sum over its blocks, in block order
      const int nb = d.cp.nb, c0 = (c / nb) * nb;
      t = 0.0;
      for (int i = 0; i < nb; ++i) t += colsum[c0 + i];
    }
    dot_finalize_column(d, c, t);
  }
  __syncthreads();
  dot_finalize_rhs(d, colsum);
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();  // the block may go on to reuse the shared scratch
}

// Two-level variant for the batched kernels (see BDot): any number of items
// per problem, each reduction stage reading at most 32 lines per column.
template <int CPT>
__device__ __forceinline__ void block_dot2(const DotArgs& d, double (&part)[CPT], int c0, bool has_cols, int rloc,
                                           int rows_pb, int S, int C, double* sm, int slot, const BDot& bd) {
  const bool pow2 = (S & (S - 1)) == 0 && S <= 32;
  int lines;
  if (pow2) {
    for (int off = S; off < 32; off <<= 1) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) part[q] += __shfl_xor_sync(0xffffffffu, part[q], off);
    }
    lines = kBlock / 32;
    const int lane = threadIdx.x & 31;
    if (has_cols && lane < S) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) sm[(threadIdx.x >> 5) * C + c0 + q] = part[q];
    }
  } else {
    lines = rows_pb;
    if (has_cols) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) sm[rloc * C + c0 + q] = part[q];
    }
  }
  __syncthreads();
  const int slices = blockDim.x / C;
  double* red = sm + lines * C;  // [slices][C]
  // sum `count` lines of `src` (stride C) into red, then red over slices -> out
  auto reduce_lines = [&](const double* src, int count, bool global_src, double* out) {
    if ((int)threadIdx.x < slices * C) {
      const int c = threadIdx.x % C, sl = threadIdx.x / C;
      double t0 = 0.0, t1 = 0.0;
      int r = sl;
      for (; r + slices < count; r += 2 * slices) {
        t0 += global_src ? __ldcg(src + (int64_t)r * C + c) : src[r * C + c];
        t1 += global_src ? __ldcg(src + (int64_t)(r + slices) * C + c) : src[(r + slices) * C + c];
      }
      if (r < count) t0 += global_src ? __ldcg(src + (int64_t)r * C + c) : src[r * C + c];
      red[sl * C + c] = t0 + t1;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      double t = 0.0;
      for (int sl = 0; sl < slices; ++sl) t += red[sl * C + c];
      out[c] = t;
    }
  };
  reduce_lines(sm, lines, false, bd.partials + (int64_t)slot * C);
  __threadfence();
  __syncthreads();
  __shared__ unsigned last_chunk, last_all;
  const int chunk = slot >> 5;
  const int nch = (bd.nslots + 31) >> 5;
  const int in_chunk = min(32, bd.nslots - chunk * 32);
  if (threadIdx.x == 0) last_chunk = (atomicAdd(bd.chunk_tickets + chunk, 1u) == (unsigned)in_chunk - 1u) ? 1u : 0u;
  __syncthreads();
  if (!last_chunk) return;
  __threadfence();
  reduce_lines(bd.partials + (int64_t)chunk * 32 * C, in_chunk, true, bd.chunk_partials + (int64_t)chunk * C);
  if (threadIdx.x == 0) bd.chunk_tickets[chunk] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_all = (atomicAdd(bd.ticket, 1u) == (unsigned)nch - 1u) ? 1u : 0u;
  __syncthreads();
  if (!last_all) return;
  __threadfence();
  double* colsum = sm;  // [C] (the line area is free now)
  reduce_lines(bd.chunk_partials, nch, true, colsum);
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) dot_finalize_column(d, c, colsum[c]);
  __syncthreads();
  dot_finalize_rhs(d, colsum);
  if (threadIdx.x == 0) *bd.ticket = 0u;
  __syncthreads();
}

}  // namespace amgsym
