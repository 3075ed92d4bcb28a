// Finest-level products in the diagonal-offset form as a z-marching stencil.
//
// The finest-level matrices of a structured grid -- the reduced operator A^
// (eq. "hL_splitting": I (x) A_inn plus the interface couplings) and the
// FSAI factors G, G^T of A_inn -- have their entries on the diagonals
// {0, +-1, +-gx, +-gxy} of the row index (gx, gxy: the strides of the second
// and third grid index).  The diagonal-offset kernel reads, for every row,
// the X rows row + offset through L1: seven 32-byte gathers per row, two
// batches of dependent round trips.  Here a block owns a tile of kZTX x kZTY
// consecutive (first, second index) positions and marches along the third
// index: the plane of X under the tile, with its one-point halo, is staged in
// shared memory once and read there by the neighbours, the X rows one plane
// below and above stay in registers, and the next plane's X rows and halo
// (and matrix values) are loaded while the current plane is computed.  Each X row is read about
// 1.3 times instead of 7, and a plane costs one round trip.
//
// Every neighbour is addressed by its row index (row + offset, zero outside
// [0, rows)), exactly as the diagonal-offset kernel does, so for ANY matrix
// whose offsets lie in that set -- a true grid or not -- each row's sum has
// the same terms in the same (ascending offset) order: the products are
// bit-identical to the diagonal-offset kernel's.  A fused dot's per-thread
// partials cover other rows than there, so the dot agrees to rounding.
//
// Work split: the (tile, plane) units, tile-major, are cut into one equal
// range per resident block (one wave, balanced to one plane); a range that
// crosses a tile restarts the march.  Interface rows (HAS_IFACE) follow the
// design of spmm_tile: the march stores none of them, then they are
// recomputed with their couplings from the compact list of flagged rows.
//
// Selected by opts.zmarch, off by default: at 256^3 (base block 128^3, 8 FP32
// columns) it ran the finest-level G in 39-41 us against 33 us for the
// diagonal-offset kernel.  At 110-128 registers two blocks fit an SM, 512
// rows in flight, and each plane waits one round trip and a barrier; the
// diagonal-offset kernel keeps as many rows in flight with no barrier.
#pragma once

#include "spmm_common.cuh"

namespace amgsym {

constexpr int kZTX = 32;                // tile positions along the first grid index
constexpr int kZTY = kBlock / kZTX;     // ... along the second (8)
constexpr int kZPW = kZTX + 2, kZPH = kZTY + 2;  // staged plane with its halo

// Diagonal kinds, in ascending offset order: -gxy, -gx, -1, 0, +1, +gx, +gxy.
// KM (template) is the set present: 0x7F (A), 0x0F (lower factor G), 0x78 (G^T).
constexpr int kKindAll = 0x7F, kKindLower = 0x0F, kKindUpper = 0x78;

__host__ __device__ inline size_t stencil_smem_bytes(int C, int xbytes, bool dot) {
  const size_t d = dot ? ((size_t)dot_smem_doubles(1, kBlock, C) * 8 + 31) / 32 * 32 : 0;
  return d + 2 * (size_t)kZPH * kZPW * (size_t)(C * xbytes);
}

template <typename MT, typename XT, typename OT, int CPT, int KM, bool HAS_DOT, bool HAS_IFACE>
__global__ void __launch_bounds__(kBlock, 2) stencil_kernel(SpmmArgs a) {
  using CT = typename ComputeOf<MT, XT>::type;
  using DT = typename AccOf<XT>::type;
  using V = Vec<XT, CPT>;
  if (a.skip && *a.skip == 0) return;  // uniform over the grid
  extern __shared__ __align__(32) unsigned char zsm_raw[];
  double* dsm = reinterpret_cast<double*>(zsm_raw);
  V* plane = reinterpret_cast<V*>(zsm_raw + (stencil_smem_bytes(CPT, (int)sizeof(XT), HAS_DOT) -
                                             2 * (size_t)kZPH * kZPW * sizeof(V)));
  constexpr bool KM3 = (KM >> 0) & 1, KL3 = (KM >> 1) & 1, KW = (KM >> 2) & 1;
  constexpr bool KE = (KM >> 4) & 1, KU3 = (KM >> 5) & 1, KP3 = (KM >> 6) & 1;
  const int rows = a.rows, gx = a.gx, gxy = a.gxy;
  const int nz = rows / gxy, tiles_x = gx / kZTX, tiles = tiles_x * (gxy / gx / kZTY);
  const int tx = threadIdx.x % kZTX, ty = threadIdx.x / kZTX;
  const XT* __restrict__ X = static_cast<const XT*>(a.X);
  const MT* __restrict__ dv = static_cast<const MT*>(a.dval);
  const int64_t n = a.dstride;
  // value source of each kind: its diagonal index (offsets ascending)
  int dk[7];
  {
    int d = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      dk[k] = d;
      if ((KM >> k) & 1) ++d;
    }
  }
  auto ldc = [&](int64_t j) {  // X row j, zero outside [0, rows)
    V v;
    if ((uint64_t)j < (uint64_t)rows) {
      v = ldv<XT, CPT>(X + j * CPT);
    } else {
#pragma unroll
      for (int q = 0; q < CPT; ++q) v.v[q] = (XT)0;
    }
    return v;
  };
  auto mval = [&](int k, int row) {  // value of kind k in row (0 when the column is outside)
    const int d = dk[k];
    const int64_t j = (int64_t)row + a.doff[d];
    return (uint64_t)j < (uint64_t)rows ? cvt<CT>(dv[(int64_t)a.dsrc[d] * n + row + a.dshift[d]]) : (CT)0;
  };
  // halo duty: threads 0..79 load one halo position per plane
  //   0..7 left (-1) of row ty, 8..15 right (+1), 16..47 below (-gx) of column tx, 48..79 above (+gx)
  const int h = threadIdx.x;
  int hslot = -1, hoff = 0, hx = 0, hy = 0;
  if (h < kZTY) {
    if (KW) { hslot = (h + 1) * kZPW + 0; hoff = -1; hx = 0; hy = h; }
  } else if (h < 2 * kZTY) {
    if (KE) { hslot = (h - kZTY + 1) * kZPW + kZTX + 1; hoff = 1; hx = kZTX - 1; hy = h - kZTY; }
  } else if (h < 2 * kZTY + kZTX) {
    if (KL3) { hslot = 0 * kZPW + (h - 2 * kZTY) + 1; hoff = -gx; hx = h - 2 * kZTY; hy = 0; }
  } else if (h < 2 * kZTY + 2 * kZTX) {
    if (KU3) { hslot = (kZTY + 1) * kZPW + (h - 2 * kZTY - kZTX) + 1; hoff = gx; hx = h - 2 * kZTY - kZTX; hy = kZTY - 1; }
  }
  DT dpart[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) dpart[q] = (DT)0;

  int it = 0;  // planes done by this block: the staging buffer alternates across restarts too
  const int64_t units = (int64_t)tiles * nz;
  int64_t u = units * blockIdx.x / gridDim.x;
  const int64_t u_end = units * (blockIdx.x + 1) / gridDim.x;
  while (u < u_end) {  // block-uniform
    const int tile = (int)(u / nz);
    const int zs = (int)(u - (int64_t)tile * nz);
    const int64_t zrem = (int64_t)zs + (u_end - u);
    const int ze = zrem < nz ? (int)zrem : nz;
    u += ze - zs;
    const int x0 = (tile % tiles_x) * kZTX, y0 = (tile / tiles_x) * kZTY;
    const int base = x0 + tx + gx * (y0 + ty);      // this thread's row on plane 0
    const int hbase = x0 + hx + gx * (y0 + hy) + hoff;  // its halo row on plane 0
    V xm, xc, xn, hv;
    if (KM3) xm = ldc((int64_t)base + (int64_t)gxy * (zs - 1));
    xc = ldc((int64_t)base + (int64_t)gxy * zs);
    xn = ldc((int64_t)base + (int64_t)gxy * (zs + 1));
    if (hslot >= 0) hv = ldc((int64_t)hbase + (int64_t)gxy * zs);
    CT m[7];  // this plane's values, loaded one plane ahead
#pragma unroll
    for (int k = 0; k < 7; ++k)
      if ((KM >> k) & 1) m[k] = mval(k, base + gxy * zs);
    for (int z = zs; z < ze; ++z) {
      V* P = plane + (it++ & 1) * (kZPH * kZPW);
      P[(ty + 1) * kZPW + tx + 1] = xc;
      if (hslot >= 0) P[hslot] = hv;
      // next plane: the X rows two planes up and the halo one plane up
      V xnn, hvn;
      CT mn[7];
      if (z + 1 < ze) {
        xnn = ldc((int64_t)base + (int64_t)gxy * (z + 2));
        if (hslot >= 0) hvn = ldc((int64_t)hbase + (int64_t)gxy * (z + 1));
#pragma unroll
        for (int k = 0; k < 7; ++k)
          if ((KM >> k) & 1) mn[k] = mval(k, base + gxy * (z + 1));
      }
      const int row = base + gxy * z;
      // this plane's epilogue operands, in flight across the barrier
      V zpre, wpre;
      const bool use_z = a.beta != 0.0, use_w = HAS_DOT && a.dot.mode == DOT_WY;
      if (use_z) zpre = ldv<XT, CPT>(static_cast<const XT*>(a.Z) + (int64_t)row * CPT);
      if (use_w) wpre = ldv<XT, CPT>(static_cast<const XT*>(a.dot.W) + (int64_t)row * CPT);
      const uint32_t iface_word = HAS_IFACE ? __ldg(a.imask + (row >> 5)) : 0u;
      __syncthreads();
      CT acc[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = (CT)0;
      auto add = [&](CT mk, const V& xv) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = fma(mk, (CT)xv.v[q], acc[q]);
      };
      if (KM3) add(m[0], xm);
      if (KL3) add(m[1], P[ty * kZPW + tx + 1]);
      if (KW) add(m[2], P[(ty + 1) * kZPW + tx]);
      add(m[3], xc);
      if (KE) add(m[4], P[(ty + 1) * kZPW + tx + 2]);
      if (KU3) add(m[5], P[(ty + 2) * kZPW + tx + 1]);
      if (KP3) add(m[6], xn);
      const bool flagged = HAS_IFACE && ((iface_word >> (row & 31)) & 1u);
      if (!flagged) row_epilogue<XT, OT, CT, DT, CPT, HAS_DOT, false>(a, row, 0, acc, zpre, use_z, wpre, use_w, dpart);
      if (KM3) xm = xc;
      xc = xn;
      xn = xnn;
      hv = hvn;
#pragma unroll
      for (int k = 0; k < 7; ++k) m[k] = mn[k];
    }
  }
  if (HAS_IFACE) {
    // the flagged rows, with their couplings (the second pass of spmm_tile)
    for (int f = blockIdx.x * kBlock + threadIdx.x; f < a.nflag; f += gridDim.x * kBlock) {
      const int row = __ldg(a.irows + f);
      CT acc[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = (CT)0;
      dia_row<MT, XT, CT, CPT, false>(a, row, 0, acc);
      iface_row<XT, CT, CPT, false>(a, f, 0, acc);
      row_epilogue<XT, OT, CT, DT, CPT, HAS_DOT, false>(a, row, 0, acc, V{}, false, V{}, false, dpart);
    }
  }
  if (HAS_DOT) {
    double part[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) part[q] = (double)dpart[q];
    block_dot<CPT>(a.dot, part, 0, true, threadIdx.x, kBlock, 1, a.C, dsm, blockIdx.x, gridDim.x, a.dot.sc.partials,
                   a.dot.sc.ticket);
  }
}

}  // namespace amgsym
