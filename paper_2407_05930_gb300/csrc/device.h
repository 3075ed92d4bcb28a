// Device-side types and kernel launchers shared by the .cu translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <vector>

#include "internal.h"

namespace amgsym {

// Matrix value storage of a device matrix.
enum ValType { VAL_F64 = 0, VAL_F32 = 1, VAL_BF16 = 2 };
// Vector storage.
enum VecType { VEC_F64 = 0, VEC_F32 = 1 };

// CSR on the device with 32-bit row pointers and columns; one value array
// per precision that was built.
struct DevCsr {
  int32_t rows = 0, cols = 0;
  int64_t nnz = 0;
  double avg_row = 0.0;  // nnz / rows (tile heuristic)
  int32_t* ptr = nullptr;
  int32_t* idx = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  __nv_bfloat16* v16 = nullptr;
  const void* vals(ValType t) const {
    return t == VAL_F64 ? (const void*)v64 : t == VAL_F32 ? (const void*)v32 : (const void*)v16;
  }
  // Diagonal-offset copy (ndiag > 0; indexing as the host Dia): [nstored]
  // value arrays of dstride >= rows elements (rows rounded up to 8, zero
  // padded, so every array starts 16-byte aligned) per precision built.
  int64_t dstride = 0;
  int32_t ndiag = 0;
  int32_t doff[kMaxDiag] = {}, dsrc[kMaxDiag] = {}, dshift[kMaxDiag] = {};
  double* dv64 = nullptr;
  float* dv32 = nullptr;
  __nv_bfloat16* dv16 = nullptr;
  const void* dvals(ValType t) const {
    return t == VAL_F64 ? (const void*)dv64 : t == VAL_F32 ? (const void*)dv32 : (const void*)dv16;
  }
  // Halo-staged form (htiles > 0): tiles of hrows consecutive rows; tile t
  // reads the X rows hx[hptr[t] .. hptr[t+1]) (sorted, hmax at most, hsum in
  // all), and entry k's column is hx[hptr[t] + lidx[k]].  Values and row
  // pointers are the CSR arrays above.
  int32_t htiles = 0, hrows = 0, hmax = 0;
  int64_t hsum = 0;
  int32_t* hptr = nullptr;
  int32_t* hx = nullptr;
  uint16_t* lidx = nullptr;
  // Sliced form (nslices > 0; SELL-32 with windowed row sorting): slice s
  // holds the rows srow[32 s .. 32 s + 32) (-1: none), each row's entries in
  // its CSR order, column-major: entry e of slot l at sptr[s] + 32 e + l
  // (sidx -1 past the row's end).  Rows are sorted by length, longest first,
  // within windows of kSellWindow rows, so a slice's width is close to its
  // rows' lengths.  One value array per precision built.
  int32_t nslices = 0;
  int64_t sentries = 0;
  int32_t* sptr = nullptr;
  int32_t* srow = nullptr;
  int32_t* sidx = nullptr;
  double* sv64 = nullptr;
  float* sv32 = nullptr;
  __nv_bfloat16* sv16 = nullptr;
  const void* svals(ValType t) const {
    return t == VAL_F64 ? (const void*)sv64 : t == VAL_F32 ? (const void*)sv32 : (const void*)sv16;
  }
};
constexpr int kSellWindow = 256;

// Interface couplings A_out,i of eq. "hL_splitting" in a form the SpMM can
// look up per row at ~0.25 byte per row: a bit per row (is there any
// coupling?) and, per 32-row word, the number of flagged rows before it.
struct DevIface {
  int32_t n_rows_flagged = 0;
  int64_t n_entries = 0;
  uint32_t* mask = nullptr;    // ceil(n_b / 32)
  int32_t* prefix = nullptr;   // ceil(n_b / 32)
  int32_t* iptr = nullptr;     // n_rows_flagged + 1
  int32_t* irows = nullptr;    // n_rows_flagged: the flagged rows, ascending
  int32_t* icol = nullptr;     // n_entries
  double* ival64 = nullptr;    // n_entries * nb
  float* ival32 = nullptr;     // n_entries * nb
};

struct DevLevel {
  int32_t n = 0;
  DevCsr A, P, R, G, Gt;
  double omega = 1.0;
  double* cinv = nullptr;  // coarsest: dense inverse, FP64 row-major n x n
  // Diagonal G (an FSAI pattern of one entry per row): the smoother omega G^T G
  // is the diagonal jd = omega g_ii^2, applied elementwise (damped Jacobi).
  double* jd64 = nullptr;
  float* jd32 = nullptr;
  const void* jd(VecType t) const { return t == VEC_F64 ? (const void*)jd64 : (const void*)jd32; }
};

// Per-column CG scalars and solve status (device).
struct DevScalars {
  double* rz = nullptr;      // <r, z> per column
  double* alpha = nullptr;
  double* beta = nullptr;
  double* rr = nullptr;      // <r, r> per column (last computed)
  double* bnorm2 = nullptr;  // ||b^||^2 per RHS (reference for the stopping test)
  double* relres = nullptr;  // per RHS
  double* tol2 = nullptr;    // squared relative-residual target (device scalar)
  int32_t* active = nullptr; // per column: 1 while its RHS has not converged
  int32_t* status = nullptr; // [0] active RHS count, [1] breakdown flag, [2] iterations
  double* partials = nullptr;  // dot-product block partials
  unsigned* ticket = nullptr;  // last-block counter
  int64_t partial_cap = 0;     // doubles available in partials
};

// Shape block for the convergence finalisation (the tolerance itself is the
// device scalar DevScalars::tol2, so captured graphs do not depend on it).
struct ConvParams {
  int32_t nrhs, nb;  // columns = nrhs * nb
  int32_t count_iter;
};

// Dot-product finalisation modes (executed by the last block of a kernel).
enum DotFinal {
  FIN_NONE = 0,
  FIN_STORE_RZ = 1,  // rz[c] = sum
  FIN_ALPHA = 2,     // alpha[c] = active ? rz[c] / sum : 0 ; breakdown check
  FIN_BETA = 3,      // beta[c] = active ? sum / rz[c] : 0 ; rz[c] = sum
  FIN_CONV = 4,      // rr[c] = sum ; per-RHS relres = sqrt(sum rr)/||b|| ; deactivate converged
  FIN_STORE_BN = 5   // bnorm2[rhs] = sum over the RHS's columns
};

enum DotMode { DOT_NONE = 0, DOT_WY = 1, DOT_YY = 2 };

struct DotArgs {
  int32_t mode = DOT_NONE;
  int32_t final = FIN_NONE;
  // 1: the blocks of a right-hand side are coupled (a preconditioner that is
  // not block diagonal in the transformed basis, AMGR): the CG scalars of
  // every column come from the sum over its RHS's 2^s columns (one CG per RHS)
  int32_t coupled = 0;
  const void* W = nullptr;  // partner vector for DOT_WY (XT layout [rows][C])
  DevScalars sc;
  ConvParams cp{};
};

struct SpmmArgs {
  int32_t rows = 0, C = 0;
  const int32_t* ptr = nullptr;
  const int32_t* idx = nullptr;
  const void* val = nullptr;
  const void* X = nullptr;
  void* Y = nullptr;
  const void* Z = nullptr;  // epilogue operand (XT)
  double alpha = 1.0, beta = 0.0;
  // Interface correction (NULL mask = none).
  const uint32_t* imask = nullptr;
  const int32_t* iprefix = nullptr;
  const int32_t* iptr = nullptr;
  const int32_t* irows = nullptr;  // flagged rows, ascending (the second pass)
  int32_t nflag = 0;
  const int32_t* icol = nullptr;
  const void* ival = nullptr;  // same precision class as the accumulation
  int32_t nb = 1;
  // Early exit: when non-NULL and *skip == 0 (no active RHS) the kernel does
  // nothing (lets the host run one iteration ahead of its convergence check).
  const int32_t* skip = nullptr;
  // Tile: entry lanes per row (1, 2, 4, 8, 16; 0 = 1) and columns per
  // thread (0 = one 16-byte vector; 2x that when C allows); see spmm_kernel.
  int32_t kl = 0;
  int32_t cpt = 0;
  // Diagonal-offset form (ndiag > 0 selects it; ptr/idx/val unused): the
  // entry (row, row + doff[d]) exists when that column is in [0, rows) and
  // has the value dval[dsrc[d] * dstride + row + dshift[d]].
  int32_t ndiag = 0;
  int32_t doff[kMaxDiag] = {}, dsrc[kMaxDiag] = {}, dshift[kMaxDiag] = {};
  int64_t dstride = 0;
  const void* dval = nullptr;
  // z-marching stencil form of a diagonal-offset matrix (stencil.cuh): its
  // offsets are {0, +-1, +-gx, +-gxy} (gkm: the set, 0 = not eligible)
  int32_t gx = 0, gxy = 0, gkm = 0;
  // Diagonal-smoother epilogues (levels whose G is diagonal, jd = w g_ii^2,
  // vector precision): jmode 1 also writes Y2 = jd o Y (presmoothing of the
  // next level fused into its restriction); jmode 2 writes Y = X + jd o
  // (alpha A X + beta Z) instead of the residual itself (postsmoothing fused
  // into its residual; Y must not alias X).
  int32_t jmode = 0;
  const void* jd = nullptr;
  void* Y2 = nullptr;
  // Halo-staged form of a CSR matrix (htiles > 0; see DevCsr): used by
  // launch_spmm for products without a dot or interface when the largest halo
  // fits the shared-memory limit, else the CSR kernel runs.
  int32_t htiles = 0, hrows = 0, hmax = 0;
  const int32_t* hptr = nullptr;
  const int32_t* hx = nullptr;
  const uint16_t* lidx = nullptr;
  // Sliced form of a CSR matrix (nslices > 0; see DevCsr): used by
  // launch_spmm for products without a dot or interface at one vector of C
  // columns per thread with at most 4 entry lanes, else the CSR kernel runs.
  int32_t nslices = 0;
  const int32_t* sptr = nullptr;
  const int32_t* srow = nullptr;
  const int32_t* sidx = nullptr;
  const void* sval = nullptr;
  DotArgs dot;
};

// Launchers (k_spmm.cu).  mt: matrix values, xt: X/Z/W vectors, ot: Y.
void launch_spmm(ValType mt, VecType xt, VecType ot, const SpmmArgs& a, cudaStream_t st);
// The (columns per thread, entry lanes) launch_spmm runs for these arguments.
void spmm_resolved_tile(VecType xt, VecType ot, const SpmmArgs& a, int* cpt, int* kl);
// Whether launch_spmm runs the halo-staged kernel for these arguments.
bool spmm_uses_halo(VecType xt, const SpmmArgs& a);
// Whether launch_spmm runs the sliced (SELL) kernel for these arguments.
bool spmm_uses_sell(VecType xt, VecType ot, const SpmmArgs& a);
// Whether launch_spmm runs the z-marching stencil kernel for these arguments.
bool spmm_uses_stencil(ValType mt, VecType xt, VecType ot, const SpmmArgs& a);
// The stencil form of a diagonal-offset matrix (offsets off[0..ndiag),
// ascending): sets gx, gxy and the offset set gkm of `a` when they fit the
// z-marching kernel's tiles (else leaves gkm = 0).
void stencil_geometry(int32_t rows, int32_t ndiag, const int32_t* off, SpmmArgs& a);

// Elementwise / transform / small kernels (k_misc.cu).
void launch_transform_fwd(const double* b, int32_t nrhs, int64_t ld, const int32_t* perm, int64_t n_b,
                          int32_t s, void* xhat, VecType ot, cudaStream_t st);
void launch_transform_bwd(const void* xhat, VecType it, int32_t nrhs, const int32_t* perm, int64_t n_b,
                          int32_t s, double* x, int64_t ld, cudaStream_t st);
// x += alpha p ; r -= alpha q ; rr = <r, r>  (finalisation FIN_CONV)
void launch_cg_update1(VecType vt, int64_t rows, int32_t C, void* x, void* r, const void* p,
                       const void* q, const DotArgs& dot, cudaStream_t st, const int32_t* skip = nullptr);
// p = z + beta p
void launch_cg_update2(VecType vt, int64_t rows, int32_t C, void* p, const void* z,
                       const double* beta, cudaStream_t st, const int32_t* skip = nullptr);
// y (f64) += x (f32 or f64)
void launch_add_to_f64(VecType xt, int64_t count, double* y, const void* x, cudaStream_t st);
void launch_copy(VecType vt, int64_t count, void* dst, const void* src, cudaStream_t st);
void launch_zero(VecType vt, int64_t count, void* dst, cudaStream_t st);
// dot over a whole [rows][C] array (for ||b^||^2 etc.)
void launch_dot(VecType vt, int64_t rows, int32_t C, const void* a, const void* b, const DotArgs& dot,
                cudaStream_t st, const int32_t* skip = nullptr);
// Z = Ainv Y (dense coarsest solve, FP64 arithmetic)
// Diagonal smoother step: z = jd o src (accumulate = 0) or z += jd o src
// (accumulate = 1), jd one value per row, src and z [rows][C].
void launch_jacobi(VecType vt, int64_t rows, int32_t C, const void* jd, const void* src, void* z, int accumulate,
                   cudaStream_t st, const int32_t* skip = nullptr);
void launch_coarse_solve(VecType vt, int32_t n, int32_t C, const double* Ainv, const void* Y, void* Z,
                         cudaStream_t st, const int32_t* skip = nullptr);
// Remove, for every RHS r, the mean of column r*nb of X ([rows][nrhs*nb],
// FP64): the constant component of the natural-order vector X represents
// (singular, pure Neumann problems).  scratch: at least (blocks + 1) * nrhs
// doubles for up to scratch_cap / nrhs - 1 blocks.
void launch_sub_block0_mean(double* X, int64_t rows, int32_t nrhs, int32_t nb, double* scratch,
                            int64_t scratch_cap, cudaStream_t st);
// Multi-vector kernels (k_krylov.cu), FP64 [rows][C] vectors; a set V of J
// vectors with stride vstride and Cv columns (column c pairs with c % Cv).
// launch_mdot: H[j * C + c] = sum_rows V_j[row][c % Cv] W[row][c] (device H,
// part: scratch of mdot_blocks(rows, C) * J * C doubles).
int mdot_blocks(int64_t rows, int32_t C);
void launch_mdot(const double* V, int64_t vstride, int32_t Cv, int32_t J, const double* W, int64_t rows, int32_t C,
                 double* part, double* H, cudaStream_t st);
// W[row][c] += sign * sum_j V_j[row][c % Cv] H[j * C + c]
void launch_maxpy(const double* V, int64_t vstride, int32_t Cv, int32_t J, const double* H, double sign, double* W,
                  int64_t rows, int32_t C, cudaStream_t st);
// out[row][c] = W[row][c] s[c] (out may be W)
void launch_colscale(const double* W, const double* s, double* out, int64_t rows, int32_t C, cudaStream_t st);
// AMGR coarse step layouts (k_misc.cu): dir 0 from the transformed
// [ncb][nrhs * nb] layout to the full coarse [ncb * nb][nrhs] layout (inverse
// butterfly, scale 1/nb), dir 1 back (forward butterfly).  nb <= 16.  dir 0
// writes alpha * (that) + beta * Z (Z in the output layout, read only when
// beta != 0).
void launch_coarse_relayout(VecType vt, const void* in, void* out, int64_t ncb, int32_t nrhs, int32_t nb, int dir,
                            cudaStream_t st, double alpha = 1.0, double beta = 0.0, const void* Z = nullptr);
// A one-thread kernel that sleeps about naps x 10 us and returns (a bounded
// loop, it waits on nothing): holds a stream while the host enqueues the
// launches behind it, so that they then run back to back (per-launch timing).
void launch_hold(int32_t naps, cudaStream_t st);
// *dst = v (a one-thread kernel, so the write is ordered on the stream and capturable)
void launch_set_value(double* dst, double v, cudaStream_t st);
// CG initial scalars: active = 1 for columns of RHS with nonzero ||b||, status reset.
void launch_init_scalars(const DevScalars& sc, int32_t nrhs, int32_t nb, cudaStream_t st);
void launch_fv_grad(int32_t d, const int64_t* N, const double* widths, const double* k, const double* u,
                    const double* lam, int32_t nrhs, int64_t ld, double* grad, int32_t accumulate,
                    cudaStream_t st);

// Host-side count of kernel launches issued by this library (graph replays
// add the number of kernels in the graph).
void count_launch(int64_t n = 1);
int64_t launch_count();

int num_sms();
int max_grid_blocks();  // blocks for grid-stride kernels (SMs x resident blocks)

// Full-wave grid for a 256-thread kernel: SMs x the blocks of this kernel
// that fit on one SM (registers, shared memory), looked up once per kernel.
int resident_grid(const void* kernel, size_t smem_bytes);

}  // namespace amgsym

namespace amgsym {

// ---------------------------------------------------------------------------
// Batched (many problems per launch) kernels: k_batch.cu.
//
// A batched launch walks a work list of items; an item is a range of rows of
// one problem's operation (its arguments at index `arg`).  Rows of an item
// start at a multiple of that problem's row-slot count, so the tile layout of
// the single-problem kernels applies unchanged.  `slot` numbers the items of
// one problem (0 .. nslots-1) for the deterministic dot reduction.
struct BItem {
  int32_t arg;
  int32_t first_slot;  // first row slot (row = slot * rows_per_block)
  int32_t row_end;
  int32_t slot;
};

// Where the dot partials of one problem's items go.  Two-level reduction:
// items write partials[slot]; the last item of each chunk of 32 slots sums
// them into chunk_partials[chunk]; the last chunk sums those and finalises.
struct BDot {
  double* partials = nullptr;        // [nslots][C]
  double* chunk_partials = nullptr;  // [ceil(nslots / 32)][C]
  unsigned* chunk_tickets = nullptr; // [ceil(nslots / 32)], zero between launches
  unsigned* ticket = nullptr;        // zero between launches
  int32_t nslots = 0;
};

// Arguments of one problem for the batched vector kernels.
struct UpdArgs {
  int32_t rows = 0, C = 0;
  void* x = nullptr;        // update1: x ; update2: p ; copy: dst ; add: y (f64) ; jacobi: z
  void* r = nullptr;        // update1: r
  const void* p = nullptr;  // update1: p ; update2: z ; copy/add: src ; jacobi: src
  const void* q = nullptr;  // update1: q
  const double* beta = nullptr;
  const int32_t* skip = nullptr;
  const void* jd = nullptr;  // jacobi: one value per row
  int32_t accumulate = 0;    // jacobi: z += jd o src instead of z = jd o src
  DotArgs dot;
};

// Dense coarsest-level solve of one problem.
struct CoarseArgs {
  int32_t n = 0, C = 0;
  const double* Ainv = nullptr;
  const void* Y = nullptr;
  void* Z = nullptr;
  const int32_t* skip = nullptr;
};

enum BatchVecOp { BOP_UPDATE1 = 0, BOP_UPDATE2 = 1, BOP_COPY = 2, BOP_JACOBI = 3 };

// ---------------------------------------------------------------------------
// Persistent coarse-cycle kernel (k_cycle.cu): the phases of the V-cycle over
// the coarsest levels, one cooperative launch, grid barriers between phases.
enum CycleKind { CYCLE_SPMM = 0, CYCLE_DENSE = 1, CYCLE_JACOBI = 2 };
// Diagonal smoother step (as launch_jacobi).
struct JacobiArgs {
  int64_t rows = 0;
  int32_t C = 0, accumulate = 0;
  const void* jd = nullptr;
  const void* src = nullptr;
  void* z = nullptr;
};
struct CyclePhase {
  int32_t kind = CYCLE_SPMM;
  SpmmArgs a;    // CYCLE_SPMM (no dot, no interface; a.kl = entry lanes)
  CoarseArgs c;  // CYCLE_DENSE
  JacobiArgs j;  // CYCLE_JACOBI
};
// Grid barrier words (device): arrivals, generation, error flag (1 = a wait
// ran out; the launch stopped early).
struct CycleBar {
  unsigned* count = nullptr;
  unsigned* gen = nullptr;
  int32_t* err = nullptr;
  unsigned extra = 0;                // arrivals awaited beyond the grid (0; 1 only in the timeout check)
  long long spins = 1ll << 22;       // polls (32 ns back-off each) before a wait gives up
};
// Columns per thread of the kernel for a column count, and its cooperative
// grid (one block per SM; 0 = unavailable).
int cycle_cpt(VecType vt, int32_t C);
int cycle_grid(ValType mt, VecType vt, int32_t C);
cudaError_t launch_cycle(ValType mt, VecType vt, int32_t C, int grid, const CyclePhase* phases, int32_t nphases,
                         const CycleBar& bar, const int32_t* skip, cudaStream_t st);

void launch_spmm_batch(ValType mt, VecType xt, VecType ot, int cpt, int kl, bool dot, bool iface, bool dia,
                       const SpmmArgs* args, const BItem* items, int32_t n_items, const BDot* dots,
                       size_t smem, cudaStream_t st);
void launch_vec_batch(int op, VecType vt, int cpt, const UpdArgs* args, const BItem* items, int32_t n_items,
                      const BDot* dots, size_t smem, cudaStream_t st);
void launch_coarse_batch(VecType vt, const CoarseArgs* args, const BItem* items, int32_t n_items, cudaStream_t st);

}  // namespace amgsym
