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

#include "spmm_common.cuh"

namespace amgsym {

template <typename MT, typename XT, typename OT, int CPT, int KL, bool HAS_DOT, bool HAS_IFACE, bool DIA>
__global__ void __launch_bounds__(kBlock, ((DIA || CPT >= 8) ? 4 : (HAS_DOT || HAS_IFACE) ? 6 : 8)) spmm_kernel(SpmmArgs a) {
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
