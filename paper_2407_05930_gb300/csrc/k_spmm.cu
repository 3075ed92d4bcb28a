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
// Matrix storage: CSR, or the diagonal-offset form of a matrix whose
// entries lie on a few diagonals (the structured-grid stencil A_inn of the
// finest level and its FSAI factors): no row pointers or column indices are
// read, the value streams and the gathered rows row + offset are contiguous
// across a warp, and a symmetric matrix reads its upper diagonals as shifted
// copies of the stored lower ones.
//
// Epilogue: Y = alpha * (M X) + beta * Z (Z read only when beta != 0), then
// an optional per-column dot (W.Y or Y.Y) reduced deterministically.
#include <cuda_bf16.h>

#include <mutex>
#include <type_traits>

#include "spmm_common.cuh"
#include "sell.cuh"
#include "stencil.cuh"

namespace amgsym {

template <typename MT, typename XT, typename OT, int CPT, int KL, bool HAS_DOT, bool HAS_IFACE, bool DIA>
__global__ void __launch_bounds__(kBlock, ((DIA && HAS_DOT) ? 3 : (DIA || CPT >= 8) ? 4 : (HAS_DOT || HAS_IFACE) ? 6 : 8)) spmm_kernel(SpmmArgs a) {
  using DT = typename AccOf<XT>::type;
  if (a.skip && *a.skip == 0) return;  // uniform over the grid
  DT dpart[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) dpart[q] = (DT)0;
  // Grid-stride over row slots: a wave of blocks sweeps one contiguous window
  // of rows, so the far neighbours one block gathers were recently brought
  // into L2 by another.
  spmm_tile<MT, XT, OT, CPT, KL, HAS_DOT, HAS_IFACE, DIA>(a, blockIdx.x, gridDim.x, a.rows, dpart);
  if (HAS_DOT) {
    const TileLayout t = tile_layout<CPT, KL>(a.C);
    extern __shared__ double sm[];
    double part[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) part[q] = (t.slot_ok && t.e == 0) ? (double)dpart[q] : 0.0;
    block_dot<CPT>(a.dot, part, t.c0, t.slot_ok && t.e == 0, t.g, t.rows_pb, t.S, a.C, sm, blockIdx.x,
                   gridDim.x, a.dot.sc.partials, a.dot.sc.ticket);
  }
}

// Halo-staged CSR product (the CSR matrices below the finest level).  The
// gathers of a coarse-level product are scattered: a warp's 32 lanes fetch
// 32-byte X rows from up to 32 different lines, and the product is bound by
// the L1 tag stage, not by DRAM.  Here the rows are cut into tiles; a block
// first copies the tile's halo -- the sorted list of X rows the tile reads --
// into shared memory with coalesced 16-byte loads (each halo row once per
// tile), then computes the tile's rows from shared memory with 16-bit local
// column indices.  The entry lanes, batches and fma order are those of the
// CSR kernel (halo_row / csr_row), so the products are bit-identical.
// Tiles are walked grid-stride by a full wave of resident blocks.
constexpr int kHaloSmemLimit = 100 * 1024;

template <typename MT, typename XT, typename OT, int CPT, int KL>
__global__ void __launch_bounds__(kBlock, 4) spmm_halo_kernel(SpmmArgs a) {
  if (a.skip && *a.skip == 0) return;  // uniform over the grid
  using CT = typename ComputeOf<MT, XT>::type;
  using DT = typename AccOf<XT>::type;
  constexpr int CH = 4;    // staging loads in flight per thread
  constexpr int MAXP = 2;  // passes of a tile whose row pointers load before the staging
  extern __shared__ __align__(16) unsigned char halo_smem[];
  XT* xs = reinterpret_cast<XT*>(halo_smem);
  const int C = a.C;
  const int TPC = C / CPT;
  const int S = TPC * KL;
  const int rows_pb = kBlock / S;
  const int g = threadIdx.x / S;
  const int w = threadIdx.x - g * S;
  const int e = KL > 1 ? w / TPC : 0;
  const int c0 = (w - e * TPC) * CPT;
  const bool slot_ok = g < rows_pb;
  const int words = C * (int)sizeof(XT) / 4;  // 32-bit words per X row
  const bool vec16 = (words & 3) == 0;
  const int q = vec16 ? words >> 2 : words;   // staged units per X row (16 or 4 bytes)
  const int32_t* __restrict__ ptr = a.ptr;
  DT dpart[CPT];
  int t = blockIdx.x;
  int hb_next = 0, he_next = 0;
  if (t < a.htiles) {
    hb_next = __ldg(a.hptr + t);
    he_next = __ldg(a.hptr + t + 1);
  }
  for (; t < a.htiles; t += gridDim.x) {
    const int h0 = hb_next, nh = he_next - hb_next;
    const int r0 = t * a.hrows, r1 = min(r0 + a.hrows, a.rows);
    // independent of the halo: this thread's row pointers of the first
    // passes, issued before the staging loads
    int kb[MAXP], ke[MAXP];
#pragma unroll
    for (int p = 0; p < MAXP; ++p) {
      const int row = r0 + p * rows_pb + g;
      kb[p] = ke[p] = 0;
      if (slot_ok && row < r1) {
        kb[p] = __ldg(ptr + row);
        ke[p] = __ldg(ptr + row + 1);
      }
    }
    const int tn = t + gridDim.x;
    if (tn < a.htiles) {
      hb_next = __ldg(a.hptr + tn);
      he_next = __ldg(a.hptr + tn + 1);
    }
    // stage the halo: CH units per thread per round, every index load of the
    // round first, then every X load, then the shared-memory stores
    const int total = nh * q;
    for (int j0 = threadIdx.x; j0 < total; j0 += kBlock * CH) {
      int col[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int j = j0 + u * kBlock;
        col[u] = j < total ? __ldg(a.hx + h0 + j / q) : 0;
      }
      if (vec16) {
        const uint4* __restrict__ X4 = static_cast<const uint4*>(a.X);
        uint4 v[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * kBlock;
          if (j < total) v[u] = __ldg(X4 + (int64_t)col[u] * q + (j - (j / q) * q));
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * kBlock;
          if (j < total) reinterpret_cast<uint4*>(halo_smem)[j] = v[u];
        }
      } else {
        const uint32_t* __restrict__ Xw = static_cast<const uint32_t*>(a.X);
        uint32_t v[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * kBlock;
          if (j < total) v[u] = __ldg(Xw + (int64_t)col[u] * q + (j - (j / q) * q));
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * kBlock;
          if (j < total) reinterpret_cast<uint32_t*>(halo_smem)[j] = v[u];
        }
      }
    }
    __syncthreads();
    int p = 0;
    for (int base = r0; base < r1; base += rows_pb, ++p) {
      const int row = base + g;
      const bool live = slot_ok && row < r1;
      CT acc[CPT];
#pragma unroll
      for (int qq = 0; qq < CPT; ++qq) acc[qq] = (CT)0;
      int b0 = 0, b1 = 0;
#pragma unroll
      for (int pp = 0; pp < MAXP; ++pp)
        if (pp == p) {
          b0 = kb[pp];
          b1 = ke[pp];
        }
      if (p >= MAXP && live) {
        b0 = __ldg(ptr + row);
        b1 = __ldg(ptr + row + 1);
      }
      if (live) halo_row<MT, XT, CT, CPT, KL>(a, xs, b0, b1, e, c0, acc);
      if (KL > 1) {
#pragma unroll
        for (int off = KL / 2; off >= 1; off >>= 1) {
#pragma unroll
          for (int qq = 0; qq < CPT; ++qq) acc[qq] += __shfl_xor_sync(0xffffffffu, acc[qq], off * TPC);
        }
      }
      if (live && e == 0)
        row_epilogue<XT, OT, CT, DT, CPT, false, false>(a, row, c0, acc, Vec<XT, CPT>{}, false, Vec<XT, CPT>{}, false,
                                                        dpart);
    }
    __syncthreads();  // the next tile overwrites the halo
  }
}

static size_t halo_smem_bytes(VecType xt, const SpmmArgs& a) {
  return (size_t)a.hmax * (size_t)a.C * (xt == VEC_F64 ? 8 : 4);
}

// The halo form pays off only with tiles enough to fill the GPU: a tile is
// one block's serial stage-then-compute, so a small level with a few dozen
// tiles runs faster as the CSR kernel's many short rows.
bool spmm_uses_halo(VecType xt, const SpmmArgs& a) {
  return a.htiles >= 2 * num_sms() && a.hptr && a.ndiag <= 0 && a.dot.mode == DOT_NONE && !a.imask &&
         halo_smem_bytes(xt, a) <= (size_t)kHaloSmemLimit;
}

template <typename MT, typename XT, typename OT, int CPT, int KL>
static void launch_h(const SpmmArgs& a, cudaStream_t st) {
  auto kern = spmm_halo_kernel<MT, XT, OT, CPT, KL>;
  const size_t smem = (size_t)a.hmax * (size_t)a.C * sizeof(XT);
  if (smem > 48 * 1024) {
    // above 48 KiB a kernel must opt in, once per device (per instantiation)
    static std::mutex mu;
    static uint64_t devices_set = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) fail(AMGSYM_ERR_CUDA, "no current device");
    std::lock_guard<std::mutex> lock(mu);
    if (!(devices_set >> dev & 1)) {
      if (cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kHaloSmemLimit) !=
          cudaSuccess)
        fail(AMGSYM_ERR_CUDA, "cannot raise the shared memory of the halo-staged SpMM");
      devices_set |= uint64_t(1) << dev;
    }
  }
  count_launch();
  const int g = std::max(1, std::min(a.htiles, resident_grid((const void*)kern, smem)));
  kern<<<g, kBlock, smem, st>>>(a);
}

template <typename MT, typename XT, typename OT, int CPT, int KL, bool DIA = false>
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
      run(spmm_kernel<MT, XT, OT, CPT, KL, true, true, DIA>, smem);
    else
      run(spmm_kernel<MT, XT, OT, CPT, KL, true, false, DIA>, smem);
  } else {
    if (ifc)
      run(spmm_kernel<MT, XT, OT, CPT, KL, false, true, DIA>, 0);
    else
      run(spmm_kernel<MT, XT, OT, CPT, KL, false, false, DIA>, 0);
  }
}

// One warp per (slice, part): C / (16-byte vector) lanes per row.
template <typename XT>
static bool sell_lanes_ok(int32_t C) {
  constexpr int v = 16 / (int)sizeof(XT);
  if (C % v) return false;
  const int tpc = C / v;
  return tpc >= 1 && tpc <= 32 && (tpc & (tpc - 1)) == 0;
}

template <typename MT, typename XT, typename OT, int KL>
static void launch_s(const SpmmArgs& a, cudaStream_t st) {
  auto kern = sell_kernel<MT, XT, OT, KL>;
  count_launch();
  const int64_t tasks = (int64_t)a.nslices * (a.C / (16 / (int)sizeof(XT)));
  const int64_t g = std::max<int64_t>(1, (tasks + kBlock / 32 - 1) / (kBlock / 32));
  if (g > INT32_MAX) fail(AMGSYM_ERR_ARG, "sliced product too large for one launch");
  kern<<<(unsigned)g, kBlock, 0, st>>>(a);
}

template <typename MT, typename XT, typename OT, int CPT>
static void launch_t(const SpmmArgs& a, cudaStream_t st) {
  if (a.ndiag > 0) {  // diagonal-offset form: one lane per row
    launch_k<MT, XT, OT, CPT, 1, true>(a, st);
    return;
  }
  const int TPC = a.C / CPT;
  // entry lanes: only with a power-of-two column-thread count, and S <= 32
  int kl = a.kl > 0 ? a.kl : 1;
  if (TPC & (TPC - 1)) kl = 1;
  while (kl > 1 && TPC * kl > 32) kl >>= 1;
  if (spmm_uses_halo(sizeof(XT) == 8 ? VEC_F64 : VEC_F32, a)) {
    switch (kl) {
      case 1: launch_h<MT, XT, OT, CPT, 1>(a, st); break;
      case 2: launch_h<MT, XT, OT, CPT, 2>(a, st); break;
      case 4: launch_h<MT, XT, OT, CPT, 4>(a, st); break;
      case 8: launch_h<MT, XT, OT, CPT, 8>(a, st); break;
      default: launch_h<MT, XT, OT, CPT, 16>(a, st); break;
    }
    return;
  }
  if (a.nslices > 0 && a.dot.mode == DOT_NONE && !a.imask && kl <= 4 && sell_lanes_ok<XT>(a.C)) {
    if (kl == 1)
      launch_s<MT, XT, OT, 1>(a, st);
    else if (kl == 2)
      launch_s<MT, XT, OT, 2>(a, st);
    else
      launch_s<MT, XT, OT, 4>(a, st);
    return;
  }
  switch (kl) {
    case 1: launch_k<MT, XT, OT, CPT, 1>(a, st); break;
    case 2: launch_k<MT, XT, OT, CPT, 2>(a, st); break;
    case 4: launch_k<MT, XT, OT, CPT, 4>(a, st); break;
    case 8: launch_k<MT, XT, OT, CPT, 8>(a, st); break;
    default: launch_k<MT, XT, OT, CPT, 16>(a, st); break;
  }
}

void stencil_geometry(int32_t rows, int32_t ndiag, const int32_t* off, SpmmArgs& a) {
  a.gx = a.gxy = a.gkm = 0;
  if (ndiag <= 0 || rows <= 0) return;
  int32_t s1 = 0, s2 = 0;  // the two distinct strides above 1
  for (int d = 0; d < ndiag; ++d) {
    const int32_t o = off[d] < 0 ? -off[d] : off[d];
    if (o <= 1 || o == s1 || o == s2) continue;
    if (!s1)
      s1 = o;
    else if (!s2)
      s2 = o;
    else
      return;
  }
  if (!s1 || !s2) return;
  const int32_t gx = std::min(s1, s2), gxy = std::max(s1, s2);
  int km = 0;
  for (int d = 0; d < ndiag; ++d) {
    const int32_t o = off[d];
    const int k = o == -gxy ? 0 : o == -gx ? 1 : o == -1 ? 2 : o == 0 ? 3 : o == 1 ? 4 : o == gx ? 5 : o == gxy ? 6 : -1;
    if (k < 0) return;
    km |= 1 << k;
  }
  if (km != kKindAll && km != kKindLower && km != kKindUpper) return;
  if (gx % kZTX || gxy % gx || (gxy / gx) % kZTY || rows % gxy) return;
  a.gx = gx;
  a.gxy = gxy;
  a.gkm = km;
}

bool spmm_uses_sell(VecType xt, VecType ot, const SpmmArgs& a) {
  if (a.nslices <= 0 || a.ndiag > 0 || a.dot.mode != DOT_NONE || a.imask || spmm_uses_halo(xt, a)) return false;
  int cpt = 0, kl = 0;
  spmm_resolved_tile(xt, ot, a, &cpt, &kl);
  return kl <= 4 && (xt == VEC_F64 ? sell_lanes_ok<double>(a.C) : sell_lanes_ok<float>(a.C));
}

bool spmm_uses_stencil(ValType mt, VecType xt, VecType ot, const SpmmArgs& a) {
  // FP32 vectors, one thread per row with all 8 columns; the interface only
  // with the full stencil (the reduced operator)
  return a.ndiag > 0 && a.gkm != 0 && xt == VEC_F32 && ot == VEC_F32 && (mt == VAL_F32 || mt == VAL_BF16) &&
         a.C == 8 && (!a.imask || a.gkm == kKindAll);
}

template <typename MT, typename XT, typename OT, int KM>
static void launch_zk(const SpmmArgs& a, cudaStream_t st) {
  const bool dot = a.dot.mode != DOT_NONE, ifc = a.imask != nullptr;
  const size_t smem = stencil_smem_bytes(8, (int)sizeof(XT), dot);
  const int64_t units = (int64_t)(a.gx / kZTX) * (a.gxy / a.gx / kZTY) * (a.rows / a.gxy);
  count_launch();
  // one wave of resident blocks, the (tile, plane) units split evenly
  auto run = [&](auto kern) {
    int g = (int)std::max<int64_t>(1, std::min<int64_t>(resident_grid((const void*)kern, smem), units));
    if (dot && (int64_t)g * a.C > a.dot.sc.partial_cap) g = (int)(a.dot.sc.partial_cap / a.C);
    kern<<<g, kBlock, smem, st>>>(a);
  };
  if constexpr (KM == kKindAll) {
    if (dot && ifc)
      run(stencil_kernel<MT, XT, OT, 8, KM, true, true>);
    else if (ifc)
      run(stencil_kernel<MT, XT, OT, 8, KM, false, true>);
    else if (dot)
      run(stencil_kernel<MT, XT, OT, 8, KM, true, false>);
    else
      run(stencil_kernel<MT, XT, OT, 8, KM, false, false>);
  } else {
    if (dot)
      run(stencil_kernel<MT, XT, OT, 8, KM, true, false>);
    else
      run(stencil_kernel<MT, XT, OT, 8, KM, false, false>);
  }
}

template <typename MT, typename XT, typename OT>
static void launch_c(const SpmmArgs& a, cudaStream_t st) {
  if constexpr (std::is_same<XT, float>::value && std::is_same<OT, float>::value && !std::is_same<MT, double>::value) {
    if (spmm_uses_stencil(std::is_same<MT, float>::value ? VAL_F32 : VAL_BF16, VEC_F32, VEC_F32, a)) {
      if (a.gkm == kKindAll)
        launch_zk<MT, XT, OT, kKindAll>(a, st);
      else if (a.gkm == kKindLower)
        launch_zk<MT, XT, OT, kKindLower>(a, st);
      else
        launch_zk<MT, XT, OT, kKindUpper>(a, st);
      return;
    }
  }
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

void spmm_resolved_tile(VecType xt, VecType ot, const SpmmArgs& a, int* cpt, int* kl) {
  // the choices of launch_c and launch_t
  const int V = std::min(16 / (xt == VEC_F64 ? 8 : 4), 16 / (ot == VEC_F64 ? 8 : 4));
  const int want = a.cpt > 0 ? a.cpt : V;
  int c;
  if (want >= 2 * V && V == 4 && a.C % 8 == 0 && a.C / 8 <= kBlock)
    c = 8;
  else if (want >= 2 * V && V == 2 && a.C % 4 == 0 && a.C / 4 <= kBlock)
    c = 4;
  else if (V >= 4 && a.C % 4 == 0 && a.C / 4 <= kBlock)
    c = 4;
  else if (V >= 2 && a.C % 2 == 0 && a.C / 2 <= kBlock)
    c = 2;
  else
    c = 1;
  int k = 1;
  if (a.ndiag <= 0) {
    const int tpc = a.C / c;
    k = a.kl > 0 ? a.kl : 1;
    if (tpc & (tpc - 1)) k = 1;
    while (k > 1 && tpc * k > 32) k >>= 1;
  }
  *cpt = c;
  *kl = k;
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
