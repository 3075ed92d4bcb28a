/*
 * amgsym.h -- C ABI of the symmetry-reduced AMG-PCG Poisson solver.
 *
 * Method: A. Alsalti-Baldellou, C. Janna, X. Alvarez-Farre, F. X. Trias,
 * "A multigrid reduction framework for domains with symmetries" (arXiv 2407.05930).
 *
 *   Sec. 2, eq. "fields_struct", Fig. "1d_case": mirrored ordering of the unknowns.
 *   Sec. 2, eq. "struct_2sym": with s reflection symmetries the operator has
 *       2^s x 2^s blocks, block (p, q) = H_{p XOR q} (0-based copies).
 *   Sec. 2, eq. "split_s": H = I_{2^s} (x) H_inn + H_out, H_inn = H_1 (0-based: H_0).
 *   Sec. 2, eq. "P_s": orthonormal change of basis, P_s^{-1} = P_s.
 *   Sec. 2, eqs. "hL_s", "hL_splitting": P_s A P_s = blockdiag(A^_i),
 *       A^_i = A_inn + A_out,i.
 *   Alg. 1 ("symsolver"): b^ = P_s b; solve A^_i x^_i = b^_i for all i; x = P_s x^.
 *   Sec. 2.2, eqs. "AMGinn", "LRCAMG" (k = 0): the preconditioner I (x) M_inn^{-1},
 *       one AMG hierarchy of A_inn applied to all 2^s blocks by SpMM.
 *   Sec. 5: PCG outer iteration; AMG = PMIS coarsening, extended+i
 *       interpolation, FSAI smoother, direct coarsest solve.
 *
 * Conventions (every entry point):
 *   - Indices are 0-based.  Copy j of the base mesh is the base reflected
 *     across every axis whose bit is set in j (copy 0 = the base itself).
 *   - "host" pointers are ordinary CPU memory; the library copies what it
 *     keeps, the caller keeps ownership.  "device" pointers are CUDA global
 *     memory of the current device, owned by the caller, and are used
 *     asynchronously on the caller's stream (`stream`, a cudaStream_t; NULL =
 *     legacy default stream).
 *   - Natural-order device vectors are FP64, `nrhs` vectors of length n with
 *     leading dimension `ld` >= n (vector r starts at ptr + r*ld).
 *   - Reduced (transformed) device arrays are interleaved: shape [n_b][c]
 *     row-major with c = nrhs * 2^s columns, column rhs*2^s + i holding block
 *     i of right-hand side rhs.  They carry the unnormalised Walsh-Hadamard
 *     transform, i.e. 2^{s/2} * P_s b (see amgsym_transform_forward).
 *   - No exception crosses the ABI.  A negative status is an error; the
 *     message is available from amgsym_last_error() (thread-local).  A
 *     positive status is a warning with valid outputs.
 *   - Not thread-safe per handle: one thread may use a handle at a time.
 */
#ifndef AMGSYM_H
#define AMGSYM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amgsym_problem* amgsym_t;

typedef enum {
  AMGSYM_OK = 0,
  AMGSYM_NOT_CONVERGED = 1,        /* warning: maxit reached, outputs valid */
  AMGSYM_ERR_ARG = -1,             /* bad argument (null pointer, size, range) */
  AMGSYM_ERR_MAP = -2,             /* symmetry map is not a bijection / bad shape */
  AMGSYM_ERR_NOT_SYMMETRIC = -3,   /* matrix violates the block structure of
                                      eq. "struct_2sym" or is not symmetric */
  AMGSYM_ERR_NOT_SPD = -4,         /* non-positive diagonal or pivot in setup */
  AMGSYM_ERR_BREAKDOWN = -5,       /* PCG breakdown (p^T A p <= 0 or NaN) */
  AMGSYM_ERR_CUDA = -6,            /* CUDA runtime error */
  AMGSYM_ERR_OOM = -7,             /* host or device allocation failed */
  AMGSYM_ERR_DEVICE_TIMEOUT = -8,  /* a bounded device-side wait gave up */
  AMGSYM_ERR_STATE = -9            /* call out of order (e.g. solve before setup) */
} amgsym_status;

/* Arithmetic of a solve. */
enum {
  AMGSYM_PREC_FP64 = 0,       /* FP64 vectors, matrices, V-cycle and PCG */
  AMGSYM_PREC_MIXED_FP32 = 1, /* FP64 iterative refinement around an inner PCG
                                 with FP32 vectors and FP32 matrix values; FP64
                                 CG scalars, dot-product accumulation and
                                 coarsest solve */
  AMGSYM_PREC_MIXED_BF16 = 2  /* as MIXED_FP32, but the V-cycle's matrices
                                 (A_l for l >= 0, G, G^T, P, R) stored as BF16
                                 values, computed in FP32 */
};

/* AMG setup parameters (Sec. 5; the paper does not fix theta, omega, the
 * coarse size or the FSAI pattern for this path -- these are defaults). */
typedef struct {
  double strength_theta;    /* classical strength threshold, default 0.25 */
  double interp_trunc;      /* drop interpolation weights < trunc * row max, 0.2 */
  int32_t interp_max_elems; /* keep at most this many weights per row, 3 */
  int32_t max_levels;       /* hierarchy depth limit, 25 */
  int32_t coarse_max;       /* dense direct solve at or below this size, 256 */
  int32_t fsai_max_lower;   /* FSAI pattern: strongest lower entries per row,
                               diagonal included, default 4 (the full lower
                               pattern of a 7-point stencil) */
  double omega_scale;       /* smoother damping omega = omega_scale / lambda_max(G A G^T), 1.2 */
  int32_t nu;               /* V(nu, nu) cycle, default 1 */
  int32_t precisions;       /* bit mask of device copies to build:
                               1 = FP64, 2 = FP32, 4 = BF16 (default 3) */
  int32_t host_only;        /* 1: build the hierarchy on the host only, no
                               device upload (hierarchy export / CPU tests) */
  uint64_t seed;            /* PMIS random tie-breaking, default 12345 */
  double coarse_drop;       /* sparsified Galerkin operators below the finest level:
                               drop a_ij with |a_ij| < coarse_drop sqrt(a_ii a_jj),
                               adding it to a_ii (0 = exact Galerkin), default 0.003 */
  int32_t dia_max_diag;     /* device storage of A_l, G_l, G_l^T: a matrix whose entries
                               lie on at most this many diagonals (column offsets j - i),
                               with at most 25 % padding, is also stored by diagonals and
                               its products read no column indices (a structured-grid
                               stencil: 7 diagonals in 3-D, 4 for its FSAI factor).  An
                               exactly symmetric one stores its lower half only.  The sums
                               run in the CSR order, so results are bit-identical to the
                               CSR kernels.  0 = CSR only; default 8 = AMGSYM_MAX_DIAG */
  int32_t fuse_rows;        /* the V-cycle from the first level below the finest with at
                               most this many rows down to the coarsest solve runs as one
                               persistent cooperative kernel (grid barriers between its
                               products, the same tile code and summation order as one
                               launch per product); 0 = one launch per product.  Not used
                               by amgsym_vcycle_noalloc nor the batched solve.  Default 0:
                               on GB300 a grid barrier costs about what a kernel node of
                               the captured PCG iteration costs, so fusing gained nothing */
  int32_t fsai_max_lower_coarse; /* FSAI pattern on the levels below the finest (as
                               fsai_max_lower); 1 = diagonal, i.e. damped Jacobi with the
                               same omega rule.  Default 1: at 256^3 it gave 80 inner
                               iterations at 0.91 ms against 78 at 0.97 ms with 4 */
  int32_t halo_kb;          /* halo-staged products: the CSR matrices below the finest level
                               (A_l for l >= 1, P_l, R_l) are also cut into tiles of
                               consecutive rows, each with the sorted list of the X rows it
                               reads (its halo) and 16-bit column indices into that list;
                               a product stages a tile's halo in shared memory once and
                               gathers from there instead of through L1.  The tile height is
                               the largest of 256, 128, 64, 32 rows whose largest halo takes
                               at most halo_kb KiB at 8 FP32 columns; a launch whose halo
                               would exceed 100 KiB of shared memory (many columns, FP64)
                               runs the CSR kernel.  Same entry and lane order as the CSR
                               kernel, so results are bit-identical.  0 = CSR only
                               (default) */
  int32_t amgr;             /* 1: also build AMGR (Sec. 3.2), the paper's multigrid
                               reduction, for solves with preconditioner AMGSYM_PC_AMGR:
                               populated coarsening (Alg. "popul": the interface points and a
                               maximal independent set of the inner points at distance
                               amgr_distance in the strength graph, coarse in every copy),
                               P = I (x) [W; I] with extended+i W (eq. "amgreduction"), the
                               block-FSAI top smoother of eq. "topsmoother" (FSAI of the inner
                               block K; the coarse block with a diagonal pattern) and a
                               standard AMG hierarchy of A_c = P^T A P (eq. "structAc").
                               0 (default): not built */
  int32_t amgr_distance;    /* k of MIS(T^k) in Alg. "popul", default 1: with the extended+i
                               interpolation built here, k = 2 converged in 22-26 PCG
                               iterations on the 32^3 model problem against 9-11 for k = 1
                               (the paper pairs k = 2 with DPLS + energy minimisation) */
  int32_t amgr_interp_max;  /* AMGR interpolation weights kept per row, default 4 */
  int32_t amgr_sym_ac;      /* 1 (default): the AMGR coarse problem's level-0 products with A_c
                               run in the transformed basis: A_c = P^T A P keeps the dyadic
                               structure (eq. "structAc"), so under the butterfly of eq. "P_s"
                               it is blockdiag(A^_c,i), A^_c,i = P_b^T A_inn P_b + the
                               interface couplings of block i; the product is the butterfly,
                               the reduced SpMM over the 2^s interleaved columns (the inner
                               block read once) with the coarse couplings, and the scaled
                               butterfly back fused with the residual.  The same operator to
                               rounding with about 1/2^s of the assembled A_c's matrix
                               bytes.  0 = the assembled A_c (CSR) */
  int32_t zmarch;           /* 1: a finest-level diagonal-offset product whose
                               offsets are {0, +-1, +-gx, +-gxy} (a structured grid's 7-point
                               stencil: the reduced operator A^ and A_inn, or its FSAI factors
                               G, G^T) runs as a z-marching stencil: a block stages one plane
                               of X with its halo in shared memory and walks the third grid
                               index, reading each X row about 1.3 times instead of 7.  Every
                               neighbour is addressed by its row index like the diagonal-offset
                               kernel, so the products are bit-identical to it (a fused dot
                               agrees to rounding: other rows per thread).  Used for FP32
                               vectors with 8 columns (one RHS at s = 3), gx a multiple of 32
                               and gxy / gx of 8.  0 (default) = the diagonal-offset kernel
                               only: at 256^3 the stencil form took 39-41 us for G against
                               33 us (it holds 512 rows in flight per SM at 110-128 registers
                               and waits one round trip and a barrier per plane; the
                               diagonal-offset kernel keeps as many rows in flight without
                               barriers), 71.1 ms a solve against 67.4 ms */
  int32_t sell;             /* 1: the CSR matrices of the hierarchy (A_l, R_l, G_l with 8 or
                               more entries per row on average, not in the diagonal-offset
                               form) are also stored sliced
                               (SELL-32: rows sorted by length within windows of 256 rows,
                               slices of 32 rows, each row's entries in their CSR order,
                               column-major in the slice), and a product without a dot or
                               interface at one vector of C columns per thread (8 FP32
                               columns) runs one row per lane on it: every lane of a warp
                               loads its next entries' columns in one coalesced load and keeps
                               its gathers in flight, instead of 8 rows per warp each walking
                               row pointer -> column -> gather chains.  Each row keeps the CSR
                               kernel's entry-lane partial sums and their combination order, so
                               the products are bit-identical to the CSR kernel.  Costs about
                               1.1x the CSR index and value arrays.  0 (default) = CSR only: at
                               256^3 the level-1 residual took 100 us sliced against 72 us CSR
                               (a 256-row warp-pair covers scattered rows; the CSR kernel's 8
                               neighbouring rows per warp share their gathers), 90 ms a mixed
                               solve against 67; the FP64 solve ran 254 ms against 282 */
  int32_t lambda_device;    /* 1 (default): the smoother damping's lambda_max(G A G^T) of every
                               level is estimated on the device after the upload (the host
                               estimator's steps: 30 power iterations with Rayleigh quotients
                               from the same seeded start vector, FP64 products), not by the
                               host setup; host_only setups always use the host estimator.
                               0 = host.  (Where a coarse level has no FP64 values, opts.
                               precisions without 1, its estimate stays on the host.) */
} amgsym_opts;

#define AMGSYM_MAX_DIAG 8

/* Preconditioner of a solve (amgsym_solve_opts.preconditioner). */
enum { AMGSYM_PC_AMG = 0, AMGSYM_PC_AMGR = 1 };

typedef struct {
  double tol;          /* stop when ||b - A x||_2 / ||b||_2 <= tol per RHS, 1e-8 */
  int32_t maxit;       /* max PCG iterations (FP64) / total inner iterations (mixed), 500 */
  int32_t precision;   /* AMGSYM_PREC_*, default AMGSYM_PREC_FP64 */
  int32_t use_x0;      /* 1: x_dev holds the initial guess; 0: start from zero */
  double inner_tol;    /* mixed: floor of the inner PCG relative reduction per
                          refinement step; the target of step k is
                          clamp(tol / (4 relres_k), inner_tol, 0.5), 3e-7 */
  int32_t max_outer;   /* mixed: refinement steps, 20 */
  int32_t finest_hat;  /* 1: V-cycle finest-level residuals use A^_i instead of A_inn */
  int32_t use_graph;   /* 1: capture one PCG iteration in a CUDA graph and replay it */
  int32_t preconditioner; /* AMGSYM_PC_AMG (default): I (x) M_inn^{-1}, one AMG hierarchy of
                          A_inn for all blocks (eq. "AMGinn", LRCAMG(0)); AMGSYM_PC_AMGR: the
                          AMGR V-cycle of Alg. "apply" (needs opts.amgr at setup) */
  int32_t tune;        /* 1: time the SpMM tile candidates of every matrix once per
                          column count and precision before the first PCG loop and
                          keep the fastest (results are then reproducible only for
                          the same tile choice); 0 (default): fixed tiles from the
                          row lengths, bit-reproducible from run to run */
} amgsym_solve_opts;

typedef struct {
  int32_t iters;       /* PCG iterations (FP64) or total inner iterations (mixed) */
  int32_t outer_iters; /* refinement steps (mixed), 0 for FP64 */
  int32_t converged;   /* 1 if every RHS reached tol */
  double* relres;      /* optional, caller-owned host array [nrhs]: final true
                          relative residual of every RHS */
} amgsym_solve_info;

void amgsym_opts_default(amgsym_opts* o);
void amgsym_solve_opts_default(amgsym_solve_opts* o);

/* Thread-local message of the last error raised in this thread. */
const char* amgsym_last_error(void);

/* ------------------------------------------------------------------------
 * Problem creation (host only, no CUDA call).
 *
 * amgsym_create_problem: the full n x n operator in CSR (host; rowptr
 * [n+1] int64, colidx [nnz] int32, vals [nnz] FP64, any column order) and the
 * symmetry map perm (host int32, [2^s][n/2^s] row-major): perm[j*n_b + l] =
 * natural index of local cell l of copy j (Sec. 2, eq. "fields_struct").
 * Validates that perm is a bijection (else AMGSYM_ERR_MAP) and that every
 * entry satisfies A[perm(p,l), perm(q,l')] == H_{p XOR q}[l, l'] exactly with
 * symmetric H_m (eq. "struct_2sym"; else AMGSYM_ERR_NOT_SYMMETRIC), then keeps
 * A_inn = H_0 and the interface couplings H_m, m >= 1 (eq. "split_s"), i.e.
 * memory / 2^s.  s = 0 is allowed (no symmetry, nb = 1).
 * On success *out owns the problem; release it with amgsym_destroy.
 * ---------------------------------------------------------------------- */
amgsym_status amgsym_create_problem(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                                    const double* vals, int32_t s, const int32_t* perm,
                                    amgsym_t* out);

/* 1 if every row of the problem's operator sums to zero (relative to the
 * row's magnitude, 1e-12), i.e. A 1 = 0: the pure Neumann problem of the
 * paper's model problem (Sec. 2.2).  0 otherwise, -1 for a NULL handle.
 * Such a problem is solved in the compatible sense (see amgsym_solve). */
int32_t amgsym_is_singular(amgsym_t h);

/* Sizes of a created problem (any pointer may be NULL). */
amgsym_status amgsym_problem_sizes(amgsym_t h, int64_t* n, int64_t* n_b, int32_t* s,
                                   int64_t* nnz_inn, int64_t* n_iface_rows,
                                   int64_t* n_iface_entries);

/* Host copies of A_inn (CSR, columns sorted: rowptr [n_b+1], colidx, vals [nnz_inn])
 * and of the interface couplings: for each interface entry e (sorted by row
 * then column), row[e], col[e] and the 2^s values
 * vals[e*2^s + i] = (A_out,i)[row, col] = sum_{m>=1} (-1)^{popcount(i&m)} H_m[row, col]
 * (eq. "hL_splitting").  Buffers are caller-owned and sized from
 * amgsym_problem_sizes. */
amgsym_status amgsym_get_inner_block(amgsym_t h, int64_t* rowptr, int32_t* colidx, double* vals);
amgsym_status amgsym_get_interface(amgsym_t h, int32_t* row, int32_t* col, double* vals);

/* New values for the same operator pattern (a new coefficient field k, as
 * in the adjoint's outer loop): vals host FP64 [nnz] in the order of the
 * colidx passed to amgsym_create_problem (the handle keeps that pattern: 8
 * bytes per row and 4 per stored entry).  The values are validated as in
 * amgsym_create_problem (block structure of eq. "struct_2sym", symmetry,
 * positive diagonal); a rejected update returns the same errors and leaves
 * the problem unchanged.  An accepted one replaces A_inn and the interface
 * couplings and releases the hierarchy and the device copies: call
 * amgsym_setup before the next solve (AMGSYM_ERR_STATE otherwise). */
amgsym_status amgsym_update_values(amgsym_t h, const double* vals);

/* ------------------------------------------------------------------------
 * Setup: AMG hierarchy of A_inn on the host (PMIS, extended+i interpolation
 * truncated, Galerkin R A P with R = P^T, static FSAI on the strongest lower
 * pattern, dense inverse at the coarsest level; Sec. 5), then upload of the
 * problem and hierarchy to the current CUDA device (unless opts->host_only).
 * opts may be NULL (defaults).  May be called again to rebuild.
 * ---------------------------------------------------------------------- */
amgsym_status amgsym_setup(amgsym_t h, const amgsym_opts* opts);

/* Hierarchy export (host copies, for inspection and tests).
 * amgsym_num_levels: number of levels L (level L-1 is the dense coarsest).
 * amgsym_level_sizes: rows and nnz of A_l, P_l (n_l x n_{l+1}) and G_l;
 *   P_l and G_l are absent (0) on the coarsest level.
 * amgsym_get_level_matrix: which = 0 A_l, 1 P_l, 2 G_l; CSR into caller buffers
 *   (rowptr [rows+1], colidx, vals [nnz]).  *omega receives the smoother damping. */
int32_t amgsym_num_levels(amgsym_t h);
amgsym_status amgsym_level_sizes(amgsym_t h, int32_t level, int64_t* rows, int64_t* nnz_A,
                                 int64_t* nnz_P, int64_t* cols_P, int64_t* nnz_G, double* omega);
amgsym_status amgsym_get_level_matrix(amgsym_t h, int32_t level, int32_t which,
                                      int64_t* rowptr, int32_t* colidx, double* vals);
/* Diagonal-offset form of a level matrix (opts->dia_max_diag): which = 0 A_l,
 * 2 G_l, 3 G_l^T.  *ndiag = number of diagonals (0: the matrix is CSR only),
 * *nstored = value arrays stored (fewer than *ndiag when the matrix is exactly
 * symmetric), offsets[AMGSYM_MAX_DIAG] = the column offsets ascending, zero
 * padded.  Any output may be NULL.  Errors: AMGSYM_ERR_STATE without a
 * hierarchy, AMGSYM_ERR_ARG for a bad level or which. */
amgsym_status amgsym_level_dia(amgsym_t h, int32_t level, int32_t which, int32_t* ndiag,
                               int32_t* nstored, int32_t* offsets);

/* ------------------------------------------------------------------------
 * Solve (Alg. 1): x = A^{-1} b for nrhs right-hand sides.
 * b_dev, x_dev: device FP64 natural order, [nrhs][ld].  x_dev is the initial
 * guess if sopts->use_x0, else ignored on input.  sopts may be NULL
 * (defaults).  info may be NULL; when given, the call synchronises the stream
 * and fills it.  Returns AMGSYM_NOT_CONVERGED if maxit was reached.
 * Work arrays are allocated on the device on first use for a given nrhs
 * (grow-only) and freed by amgsym_destroy.
 *
 * Singular problems (amgsym_is_singular, pure Neumann, Sec. 2.2 eq.
 * "modelproblem"): the constant vector spans the null space; only the
 * symmetric block A^_0 = A_inn + A_out,0 of the reduced system inherits it
 * (with s >= 1, A_inn itself is regular).  The solve removes the constant
 * component of b (the compatibility condition: a b with zero sum is left as
 * it is; relres is measured against the compatible part), runs the same
 * PCG -- on the consistent singular system it converges in the range of A
 * -- and returns the solution with zero mean (the minimum-norm solution).
 * The setup inverts a singular coarsest operator (s = 0) through the
 * pseudo-inverse: (A_c + a 1 1^T / m)^{-1} - 1 1^T / (a m), a its mean
 * diagonal.  Batches do not take singular problems.
 * ---------------------------------------------------------------------- */
amgsym_status amgsym_solve(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs,
                           int64_t ld, const amgsym_solve_opts* sopts, void* stream,
                           amgsym_solve_info* info);

/* ------------------------------------------------------------------------
 * LRCAMG(k) and GMRES (Sec. 2.2, Thm. "correction_nonfact", eqs. "Ydef_AMG",
 * "LRC_AMG", "LRCAMG"; the paper's Table "lrcamg" runs GMRES with it).
 *
 * amgsym_lrc_setup: for every block i, the k eigenpairs (lambda_t, u_t) of
 * X_i = M_inn^{-1} A^_i with the smallest eigenvalues, by Lanczos in the
 * A^_i inner product, all blocks at once on the device.  The search (the
 * "eigenpair search" below) keeps a basis of `steps` vectors.  The Ritz
 * vectors u_t are A^_i-orthonormal, so v_t = A^_i u_t are the left
 * eigenvectors with V^T U = I, and the correction of eq. "LRC_AMG" is
 * (I + U Theta V^T) M_inn^{-1} with Theta_t = (1 - lambda_t) / lambda_t: it
 * maps those eigenvalues of the preconditioned block to 1.  Stores U and
 * Theta V on the device (2 k n values per block set); k = 0 removes the
 * correction.  k in [0, 64], steps in [k + 2, 400], tol in (0, 1].  Needs
 * amgsym_setup; a new setup discards the correction.  Synchronises the
 * stream.
 *
 * Eigenpair search (both setups): thick-restarted Lanczos with full
 * reorthogonalisation (Wu and Simon) on a basis of `steps` vectors,
 * restarted from the max(k + 4, steps / 2) (at most steps - 2) smallest Ritz
 * vectors, until the k smallest Ritz pairs and max(4, k / 2) more (as the
 * basis allows) have residual norms <= tol * lambda (at most 200 restarts);
 * then up to 3 more such runs from new
 * random vectors kept orthogonal to every pair found (so every copy of a
 * multiple eigenvalue is found), stopping when a run finds nothing below the
 * k-th smallest value so far.  Start vectors are uniform[-1, 1] from `seed`.
 * tol = 0.1 gives the rough pairs the paper finds sufficient; small tol
 * (1e-10) gives the eigenpairs to rounding.  A block with fewer than k
 * pairs (a space smaller than k) keeps what it has (theta 0 past them).
 *
 * amgsym_lrc_values: copies the Ritz values (host, [2^s][k], block-major)
 * into theta (may be NULL) and returns k (0: no correction, -1: no device
 * problem).
 *
 * amgsym_solve_gmres: x = A^{-1} b like amgsym_solve (same vector layout,
 * transforms, singular handling), by restarted GMRES(restart) on the
 * reduced system, right-preconditioned by eq. "LRCAMG": (I + U Theta V^T)
 * (I (x) M_inn^{-1}) with use_lrc = 1, I (x) M_inn^{-1} (LRCAMG(0)) with
 * use_lrc = 0.  Every column (block of a right-hand side) runs its own
 * Arnoldi process with classical Gram-Schmidt and one reorthogonalisation;
 * it stops when every RHS meets sopts->tol (the GMRES residual estimate,
 * confirmed by the true residual at each restart) or after sopts->maxit
 * iterations.  FP64 only (sopts->precision must be AMGSYM_PREC_FP64);
 * sopts->finest_hat applies to the V-cycle.  info->iters = GMRES iterations.
 * ---------------------------------------------------------------------- */
amgsym_status amgsym_lrc_setup(amgsym_t h, int32_t k, int32_t steps, double tol, uint64_t seed, void* stream);
int32_t amgsym_lrc_values(amgsym_t h, double* theta);
amgsym_status amgsym_solve_gmres(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                 const amgsym_solve_opts* sopts, int32_t restart, int32_t use_lrc,
                                 void* stream, amgsym_solve_info* info);

/* ------------------------------------------------------------------------
 * LRCFSAI(k) (Sec. 2.1, Thm. "correction", eqs. "Ydef", "LRC", "LRCFSAI";
 * the paper's Table "lrcfsai" runs PCG with it).
 *
 * amgsym_lrcfsai_setup: for every block i, the k eigenpairs of the smallest
 * eigenvalues lambda_t of X_i = G_inn A^_i G_inn^T, where G_inn is the FSAI
 * factor of A_inn of the setup's finest level (G_inn^T G_inn ~ A_inn^{-1}),
 * by the eigenpair search of amgsym_lrc_setup in the Euclidean inner product
 * (same steps, tol, seed and ranges), all blocks at once.  For a singular
 * problem (amgsym_is_singular) the null vector G_inn^{-T} 1 of block 0 is
 * left out.  Stores Z = G_inn^T V_k and Theta Z with Theta_t = (1 -
 * lambda_t) / lambda_t on the device; k = 0 removes the correction.  Needs a
 * hierarchy of two levels or more with FP64 values.  Synchronises the
 * stream.
 * amgsym_lrcfsai_values: Ritz values (host [2^s][k]) and k, as
 * amgsym_lrc_values.
 *
 * amgsym_solve_fsai: x = A^{-1} b like amgsym_solve, by PCG on the reduced
 * system preconditioned by I (x) G_inn^T G_inn (use_lrc = 0: LRCFSAI(0)) or by
 * eq. "LRCFSAI" (use_lrc = 1), FP64, one CG per column (the preconditioner is
 * block diagonal), recurrence residual confirmed by the true residual.
 * ---------------------------------------------------------------------- */
amgsym_status amgsym_lrcfsai_setup(amgsym_t h, int32_t k, int32_t steps, double tol, uint64_t seed,
                                   void* stream);
int32_t amgsym_lrcfsai_values(amgsym_t h, double* theta);
amgsym_status amgsym_solve_fsai(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                const amgsym_solve_opts* sopts, int32_t use_lrc, void* stream,
                                amgsym_solve_info* info);

/* Adjoint solve A^T lambda = g.  A is symmetric, so this is the same reduced
 * solve; kept as its own entry point for the differentiable interface. */
amgsym_status amgsym_solve_adjoint(amgsym_t h, const double* g_dev, double* lam_dev,
                                   int32_t nrhs, int64_t ld, const amgsym_solve_opts* sopts,
                                   void* stream, amgsym_solve_info* info);

/* ------------------------------------------------------------------------
 * Individual steps of the solve (device; after amgsym_setup), for testing and
 * composition.  `prec` selects FP64 (AMGSYM_PREC_FP64: double arrays) or FP32
 * (any mixed mode: float arrays) for the reduced arrays.
 * ---------------------------------------------------------------------- */

/* Forward transform (Alg. 1, first step; eq. "P_s"):
 * xhat[l][r*2^s + i] = sum_j (-1)^{popcount(i&j)} b_r[perm(j, l)]  (= 2^{s/2} P_s b),
 * b_dev FP64 natural [nrhs][ld], xhat_dev FP64 [n_b][nrhs*2^s]. */
amgsym_status amgsym_transform_forward(amgsym_t h, const double* b_dev, int32_t nrhs, int64_t ld,
                                       double* xhat_dev, void* stream);

/* Backward transform (Alg. 1, last step; P_s^{-1} = P_s):
 * x_r[perm(j, l)] = 2^{-s} sum_i (-1)^{popcount(i&j)} xhat[l][r*2^s + i].
 * Applied to the output of amgsym_transform_forward it returns b exactly
 * up to rounding (the 2^{-s} scale undoes both unnormalised transforms). */
amgsym_status amgsym_transform_backward(amgsym_t h, const double* xhat_dev, int32_t nrhs,
                                        double* x_dev, int64_t ld, void* stream);

/* Reduced operator (eq. "hL_splitting"):
 * Y[:, c] = A_inn X[:, c] + A_out,(c mod 2^s) X[:, c] for all columns at once,
 * A_inn read once for all columns.  X, Y: [n_b][nrhs*2^s], double (prec FP64)
 * or float (mixed).  X and Y must not overlap. */
amgsym_status amgsym_apply_reduced(amgsym_t h, const void* X_dev, void* Y_dev, int32_t nrhs,
                                   int32_t prec, void* stream);

/* Preconditioner (eqs. "AMGinn", "LRCAMG" with k = 0): Z = (I (x) M_inn^{-1}) R,
 * one symmetric V(nu, nu) cycle of the A_inn hierarchy applied to every
 * column; with finest_hat = 1 the finest-level residuals use A^_i.
 * R, Z: [n_b][nrhs*2^s], double (FP64) or float (mixed); must not overlap.
 * The levels from opts->fuse_rows down run as one persistent kernel; a
 * timed-out barrier wait there (never in a correct run) is reported by the
 * next amgsym_solve on the handle. */
amgsym_status amgsym_vcycle(amgsym_t h, const void* R_dev, void* Z_dev, int32_t nrhs,
                            int32_t prec, int32_t finest_hat, void* stream);

/* Per-launch timing of one solve step, for measurement (no counterpart in
 * the paper: it reports how this library's kernels spend a step of Alg. 1).
 *
 * Runs, on `stream`, the launches of one step of amgsym_solve with precision
 * `prec`, finest_hat and `preconditioner` (AMGSYM_PC_AMG, or AMGSYM_PC_AMGR
 * after a setup with opts.amgr: the PCG start and iteration then apply AMGR,
 * whose coarse AMG launches are records too) on b_dev (device FP64 natural
 * order [nrhs][ld]):
 * the forward transform, the FP64 outer residual, in the mixed modes the
 * inner reference norm, the PCG start (one V-cycle and z -> p), ONE PCG
 * iteration (reduced SpMM with <p, q>, the x/r update with <r, r>, the
 * V-cycle with <r, z>, the p update), in the mixed modes the refinement
 * update, and the backward transform into x_dev.  A bounded one-thread hold
 * kernel (about 3 ms of sleeps; it waits on nothing) runs first, so the host
 * has enqueued the step before the GPU reaches it and the step's kernels run
 * back to back; each launch is bracketed by two CUDA events on `stream`.
 * The call synchronises the stream.  No CUDA graph is used.
 *
 * out: caller-owned host array of max_records records; record i describes
 * the i-th timed launch in stream order: the kernel template as a profiler
 * names it, its role in the step, the V-cycle level (-1 outside it), the
 * phase (0: once per solve or refinement step, 1: every PCG iteration), the
 * algorithmic bytes of the launch (matrix storage, X once, Y once, every
 * epilogue operand once) and the event-timed duration in microseconds.
 * *count receives the number of timed launches (records beyond max_records
 * are not written).  Tiny bookkeeping kernels (scalar set-up, zero fills)
 * run untimed between the records.  Errors as amgsym_solve. */
typedef struct {
  char kernel[80];
  char role[64];
  int32_t level;
  int32_t phase;
  int64_t bytes;
  double us;
} amgsym_prof_record;
amgsym_status amgsym_profile_step(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                  int32_t prec, int32_t finest_hat, int32_t preconditioner, void* stream,
                                  amgsym_prof_record* out, int32_t max_records, int32_t* count);

/* AMGR (Sec. 3.2), built by amgsym_setup with opts->amgr = 1.
 *
 * amgsym_amgr_apply: Z = M_AMGR R, one V(1,1)-cycle of Alg. "apply" for every
 * column (layout and arguments as amgsym_vcycle): block-FSAI smoothing
 * (eq. "topsmoother"), residual with A^_i, restriction by P_b^T, the coarse
 * correction through the AMG hierarchy of A_c over the full coarse domain,
 * prolongation by P_b, block-FSAI smoothing.  AMGSYM_ERR_STATE without AMGR.
 *
 * amgsym_amgr_info (host; any output may be NULL): coarse points per copy
 * (interface plus selected inner points), nonzeros of P_b and of A_c, levels
 * of A_c's hierarchy, and the splitting cf[n_b] (1 coarse, -1 fine; int8,
 * caller-owned).
 *
 * amgsym_amgr_matrix: host CSR copies (caller buffers sized from
 * amgsym_amgr_info): which = 0 P_b (n_b x n_cb; rowptr [n_b + 1]), 1 A_c
 * (n_cb 2^s square, row / column (l, j) at l * 2^s + j for coarse point l of
 * copy j; rowptr [n_cb 2^s + 1]). */
amgsym_status amgsym_amgr_apply(amgsym_t h, const void* R_dev, void* Z_dev, int32_t nrhs, int32_t prec,
                                void* stream);
amgsym_status amgsym_amgr_info(amgsym_t h, int64_t* n_coarse_per_copy, int64_t* nnz_P, int64_t* nnz_Ac,
                               int32_t* coarse_levels, int8_t* cf);
amgsym_status amgsym_amgr_matrix(amgsym_t h, int32_t which, int64_t* rowptr, int32_t* colidx, double* vals);

/* Failure check of the persistent coarse-cycle kernel (opts->fuse_rows): runs
 * it once on the library's level work arrays with a grid barrier that awaits
 * one arrival more than the grid has, so nothing releases it, and a wait bound
 * of 4096 polls (a few milliseconds).  Every block's wait runs out, sets the
 * error word and returns; the call synchronises the stream, reads the word and
 * clears the barrier.  Returns AMGSYM_OK when the timed-out wait was reported
 * (the handle stays usable), AMGSYM_ERR_CUDA when it was not or the launch
 * failed, AMGSYM_ERR_STATE when the problem has no fused coarse cycle.  No
 * counterpart in the paper: it tests this library's own bounded waits. */
amgsym_status amgsym_cycle_timeout_check(amgsym_t h, int32_t nrhs, int32_t prec, void* stream);

/* Preconditioner without allocation: the V-cycle of amgsym_vcycle (same
 * arguments, same kernels, same result), for callers that cannot let the
 * library call cudaMalloc -- e.g. a real-time loop that must not take the
 * device-wide synchronisation an allocation implies, or a process whose device
 * memory belongs to another allocator with a fixed budget.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *
 * The level vectors come from one fixed array of 32 MiB (33554432 bytes) in
 * device global memory, declared statically in the library; every GPU that
 * loads the library holds it until the process exits.  A problem whose
 * V-cycle needs more is rejected with AMGSYM_ERR_ARG and a message giving
 * both sizes.  The need is a sum over levels of vectors of n_l x nrhs*2^s
 * values, 8 bytes each in FP64 and 4 in the mixed modes, each rounded up to
 * 256 bytes: 2 vectors on the finest level (residual, smoother temporary),
 * 4 on every other level (right-hand side, solution, residual, temporary),
 * and 2 on the dense coarsest level (right-hand side, solution) -- none when
 * the finest level is itself the coarsest.
 * The entry point calls no cudaMalloc, cudaFree or other allocating routine.
 * Its first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  All calls on a device share the one array and it
 * keeps the last call's contents (every vector is written before it is read,
 * so nothing needs clearing): calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller. */
amgsym_status amgsym_vcycle_noalloc(amgsym_t h, const void* R_dev, void* Z_dev, int32_t nrhs,
                                    int32_t prec, int32_t finest_hat, void* stream);

/* ------------------------------------------------------------------------
 * Structured-grid problem generator (host): the unit cube with N[a] cells
 * per axis (d = 1..3), cell-centred finite volumes for -div(k grad u) = f,
 * homogeneous Dirichlet.  Face transmissibility t_f = area_f /
 * sum_{c in f} h_c / (2 k_c) (a boundary face has the single cell term);
 * A_pq = -t_f, A_pp = sum over faces (per-axis low+high pairs summed first).
 * Natural order, x fastest.  Stretching: eq. "tanh" (Sec. 2.2).
 * ---------------------------------------------------------------------- */

/* Cell widths of an N-cell axis: uniform (gamma = 0) or eq. "tanh" with
 * stretching gamma; for even N the upper half mirrors the lower half exactly. */
amgsym_status amgsym_grid_widths(int64_t N, double gamma, double* widths_out);

/* Number of stored entries of the 2d+1-point operator. */
int64_t amgsym_fv_nnz(int32_t d, const int64_t* N);

/* Boundary conditions of the generator: homogeneous Dirichlet on every wall
 * (the benchmark workloads), or homogeneous Neumann on every wall -- the
 * paper's model problem (Sec. 2.2, eq. "modelproblem"), whose operator is
 * singular with the constant vector as null space. */
enum { AMGSYM_BC_DIRICHLET = 0, AMGSYM_BC_NEUMANN = 1 };

/* Assemble the full operator: widths = concatenation of the d per-axis width
 * arrays (host), k = per-cell coefficient (host, natural order).  Outputs are
 * caller-owned host buffers: rowptr [n+1], colidx/vals [amgsym_fv_nnz]. */
amgsym_status amgsym_fv_assemble(int32_t d, const int64_t* N, const double* widths,
                                 const double* k, int64_t* rowptr, int32_t* colidx,
                                 double* vals);
/* The same with boundary condition bc (AMGSYM_BC_*): a Neumann wall face
 * carries no flux, so it adds nothing to the diagonal and every row sums to
 * zero.  Same pattern and entry order as amgsym_fv_assemble. */
amgsym_status amgsym_fv_assemble_bc(int32_t d, const int64_t* N, const double* widths,
                                    const double* k, int32_t bc, int64_t* rowptr,
                                    int32_t* colidx, double* vals);

/* Mirrored-ordering map for s reflection symmetries of axes 0..s-1
 * (perm as in amgsym_create_problem, host int32 [2^s][n/2^s]). */
amgsym_status amgsym_mirror_perm(int32_t d, const int64_t* N, int32_t s, int32_t* perm);

/* Adjoint gradient with respect to g = log k (device, FP64, natural order):
 * grad[c] += sum over faces f of c of (dL/dt_f) * t_f^2 h_c / (2 area_f k_c),
 * with dL/dt_f = -(lam_p - lam_q)(u_p - u_q) (interior) or -lam_p u_p
 * (boundary), summed over nrhs pairs (u_r, lam_r) with leading dimension ld.
 * widths_dev: concatenated per-axis widths (device); k_dev per cell.
 * accumulate = 0 overwrites grad_dev, 1 adds to it. */
amgsym_status amgsym_fv_grad_logk(int32_t d, const int64_t* N, const double* widths_dev,
                                  const double* k_dev, const double* u_dev,
                                  const double* lam_dev, int32_t nrhs, int64_t ld,
                                  double* grad_dev, int32_t accumulate, void* stream);

/* ------------------------------------------------------------------------
 * Batched solve (many independent problems in one pass).
 *
 * amgsym_batch_create: a batch over `count` problems that are already set up
 * on one device (amgsym_setup, hierarchies of at least two levels, the same
 * nu), with nrhs[p] right-hand sides for problem p (nrhs[p] * 2^s_p <= 256).
 * The batch references the problems; they must outlive it.  A problem of
 * the batch may be given new values and set up again (amgsym_update_values,
 * amgsym_setup): that frees the device copies the batch's launch plans and
 * captured graph point to, and the next amgsym_batch_solve notices it and
 * rebuilds them (a process-wide generation count identifies every device
 * copy).  If the problem no longer meets the conditions above (a single-level
 * hierarchy, another nu or device), that solve returns AMGSYM_ERR_STATE.
 *
 * amgsym_batch_solve: solves every problem (Alg. 1 per problem) with the
 * mixed-precision refinement of amgsym_solve (sopts->precision must be
 * AMGSYM_PREC_MIXED_FP32 or _BF16).  All problems advance in lock step: each
 * step of an inner PCG iteration (reduced SpMM, vector updates, every V-cycle
 * product, coarsest solves) is one persistent work-list launch over all
 * problems taking part in it, and one iteration is captured in a CUDA graph.
 * b_dev[p], x_dev[p]: device FP64 natural-order [nrhs[p]][n_p] (leading
 * dimension n_p).  infos: optional array of `count` records (iters = inner
 * iterations of the batch, converged and relres per problem).
 * ---------------------------------------------------------------------- */
typedef struct amgsym_batch* amgsym_batch_t;
amgsym_status amgsym_batch_create(const amgsym_t* problems, int32_t count, const int32_t* nrhs,
                                  amgsym_batch_t* out);
amgsym_status amgsym_batch_solve(amgsym_batch_t b, const double* const* b_dev, double* const* x_dev,
                                 const amgsym_solve_opts* sopts, void* stream, amgsym_solve_info* infos);
void amgsym_batch_destroy(amgsym_batch_t b);

/* SpMM tiles in use for nrhs right-hand sides and precision prec (after a
 * solve with sopts->tune = 1 these are the tuner's choices, else the fixed
 * ones): out[0..1] = (columns per thread, entry lanes) of the reduced
 * operator, then for each level l < max_levels five pairs for A_l, G_l, G_l^T,
 * R_l, P_l (0, 0 where absent).  out holds 2 + 10 * max_levels int32. */
amgsym_status amgsym_get_tiles(amgsym_t h, int32_t nrhs, int32_t prec, int32_t* out, int32_t max_levels);

/* Number of CUDA kernels this library has launched in the process so far
 * (a replayed CUDA graph counts its kernels).  Host-side counter. */
int64_t amgsym_kernel_launches(void);

void amgsym_destroy(amgsym_t h);

#ifdef __cplusplus
}
#endif

#endif /* AMGSYM_H */
