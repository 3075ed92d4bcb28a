// Sliced (SELL-32) products of the hierarchy's CSR matrices.
//
// The coarse-level products are bound by dependent round trips, not by
// bandwidth: in the CSR kernel a warp serves 8 rows (4 entry lanes each)
// and every row walks row pointer -> column indices -> X gathers, batch
// after batch.  In the sliced form (DevCsr: rows sorted by length within
// windows, slices of 32 rows, entries column-major in the slice) a warp
// serves 16 rows (2 lanes of 4 columns each at 8 FP32 columns): the lanes'
// next B entries (columns and values) arrive in B coalesced loads while the
// previous B gathers are in flight, so a slice costs about width / B + 2
// round trips.
//
// Bit-identical to the CSR kernel at the same entry-lane count KL: a row
// keeps KL partial sums, entry i going to partial i mod KL in ascending
// order, and combines them in the order of the CSR kernel's xor-shuffle
// tree ((p0 + p2) + (p1 + p3) for KL = 4), with the same values, gathers,
// fma and epilogue.  Padding slots (column -1) are skipped.
//
// Selected by opts.sell, off by default: at 256^3 (level 1: 775k rows, 19
// entries per row) the sliced residual took 100 us against 72 us for the
// CSR kernel with 4 entry lanes (without the row sorting 115 us; with one
// row per lane at 8 columns and one wave of blocks 180 us).  ncu of the
// one-row-per-lane version at 192^3: fewer sectors (8.0M against 10.3M)
// and instructions (6.5M against 14.8M) than CSR, but long-scoreboard bound
// at 22 % achieved occupancy.  The FP64 solve gains (254 ms against 282).
#pragma once

#include "spmm_common.cuh"

namespace amgsym {

// Lanes: each row is served by TPC = C / CPT lanes of CPT columns (one
// 16-byte vector each), so a warp serves 32 / TPC rows of a slice (a task);
// a block runs kBlock / 32 tasks, and the grid covers every task (the block
// scheduler balances slices of different widths).  The next batch's columns
// and values load while the current batch's gathers are in flight.
template <typename MT, typename XT, typename OT, int KL>
__global__ void __launch_bounds__(kBlock, sizeof(XT) == 8 ? 3 : 4) sell_kernel(SpmmArgs a) {
  static_assert(KL == 1 || KL == 2 || KL == 4, "1, 2 or 4 entry lanes");
  constexpr int CPT = 16 / (int)sizeof(XT);
  using CT = typename ComputeOf<MT, XT>::type;
  using DT = typename AccOf<XT>::type;
  using V = Vec<XT, CPT>;
  if (a.skip && *a.skip == 0) return;  // uniform over the grid
  constexpr int B = 4;                 // entries per lane per round trip (a multiple of KL)
  static_assert(B % KL == 0, "batch must keep entry i in partial i mod KL");
  const int C = a.C, TPC = C / CPT, rpw = 32 / TPC;
  const int lane = threadIdx.x & 31;
  const int64_t task = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  const int64_t s = task / TPC;  // slice; this warp serves its rows part * rpw .. part * rpw + rpw
  if (s >= a.nslices) return;    // whole warps (no barrier below)
  const int part = (int)(task - s * TPC);
  const int slot = part * rpw + lane / TPC;  // row slot in the slice
  const int c0 = (lane % TPC) * CPT;
  const XT* __restrict__ X = static_cast<const XT*>(a.X);
  const MT* __restrict__ sv = static_cast<const MT*>(a.sval);
  const int32_t* __restrict__ sidx = a.sidx;
  const int row = __ldg(a.srow + s * 32 + slot);
  const int b0 = __ldg(a.sptr + s), b1 = __ldg(a.sptr + s + 1);
  CT acc[KL][CPT];
#pragma unroll
  for (int k = 0; k < KL; ++k)
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[k][q] = (CT)0;
  // b1 - b0 is a multiple of 32: the batch bounds are the same for every lane
  int jn[B];
  CT mn[B];
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int pos = b0 + 32 * u + slot;
    const bool in = pos < b1;
    jn[u] = in ? __ldg(sidx + pos) : -1;
    mn[u] = in ? cvt<CT>(sv[pos]) : (CT)0;
  }
  for (int e0 = b0; e0 < b1; e0 += 32 * B) {
    int j[B];
    CT m[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      j[u] = jn[u];
      m[u] = mn[u];
    }
    V x[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j[u] >= 0) x[u] = ldv<XT, CPT>(X + (int64_t)j[u] * C + c0);
    const int e1 = e0 + 32 * B;
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int pos = e1 + 32 * u + slot;
      const bool in = pos < b1;
      jn[u] = in ? __ldg(sidx + pos) : -1;
      mn[u] = in ? cvt<CT>(sv[pos]) : (CT)0;
    }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j[u] >= 0) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[u % KL][q] = fma(m[u], (CT)x[u].v[q], acc[u % KL][q]);
      }
  }
  CT out[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    if (KL == 1)
      out[q] = acc[0][q];
    else if (KL == 2)
      out[q] = acc[0][q] + acc[KL - 1][q];
    else
      out[q] = (acc[0][q] + acc[KL / 2][q]) + (acc[1 % KL][q] + acc[(KL / 2 + 1) % KL][q]);
  }
  DT none[CPT];  // the epilogue's dot partial: no dot here
  if (row >= 0) row_epilogue<XT, OT, CT, DT, CPT, false, false>(a, row, c0, out, V{}, false, V{}, false, none);
}

}  // namespace amgsym
