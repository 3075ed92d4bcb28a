// Internal host-side types of the amgsym library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/amgsym.h"

namespace amgsym {

// Host CSR matrix with int64 row pointers (columns need not be sorted unless
// stated by the producer).
struct Csr {
  int64_t rows = 0, cols = 0;
  std::vector<int64_t> ptr;   // rows + 1
  std::vector<int32_t> idx;
  std::vector<double> val;
  int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// Error raised inside the library; converted to a status at the ABI.
struct Error {
  amgsym_status code;
  std::string msg;
};
[[noreturn]] void fail(amgsym_status code, const std::string& msg);
void set_last_error(const std::string& msg);

// Diagonal-offset form of a square matrix whose entries lie on a few
// diagonals (the stencil of a structured grid and its FSAI factors):
// diagonal d holds the entries (i, i + off[d]), offsets ascending, and its
// value at row i is val[src[d] * rows + i + shift[d]].  shift[d] = off[d]
// for an upper diagonal of an exactly symmetric matrix, read as the mirror
// image of the stored lower diagonal src[d] (a_{i,i+o} = a_{i+o,i}); every
// other diagonal is stored (shift 0).  Positions outside the pattern hold 0.
constexpr int kMaxDiag = 8;
struct Dia {
  int32_t ndiag = 0, nstored = 0;
  int32_t off[kMaxDiag] = {}, src[kMaxDiag] = {}, shift[kMaxDiag] = {};
  std::vector<double> val;  // [nstored][rows]
};
// The diagonal-offset form of M when it is square, has at most max_diag
// distinct column offsets and at most 25 % padding; else ndiag = 0.
Dia build_dia(const Csr& M, int max_diag);

// One level of the AMG hierarchy of A_inn (host copies).
struct HostLevel {
  Csr A;        // level operator (level 0: A_inn)
  Csr P;        // prolongation n_l x n_{l+1} (absent on the coarsest level)
  Csr R;        // restriction P^T
  Csr G;        // FSAI factor, lower triangular (G^T G ~ A^{-1})
  Csr Gt;       // G^T
  Dia Adia, Gdia, Gtdia;  // diagonal-offset forms (ndiag = 0: CSR only)
  double omega = 1.0;
  double lambda_max = 0.0;
  std::vector<double> coarse_inv;  // coarsest level: dense A^{-1}, row-major
};

struct HostHierarchy {
  std::vector<HostLevel> levels;
};

struct Device;  // device-resident copies and work arrays (solve.cu)

// AMGR (Sec. 3.2): the multigrid reduction of the full operator.  Populated
// coarsening (Alg. "popul"): every interface point of the base mesh (a row
// coupled to another mirror copy) and a maximal independent set of the inner
// points at distance k in the strength graph are coarse, in every copy; the
// prolongation is I (x) P_b with P_b = [W; I] (eq. "amgreduction"); the
// top-level smoother is the block FSAI of eq. "topsmoother"; the reduced
// operator A_c = P^T A P (eq. "structAc") gets a standard AMG hierarchy.
struct HostAmgr {
  std::vector<int8_t> cf;   // per base row: 1 coarse (interface or selected inner), -1 fine
  int32_t n_cb = 0;         // coarse points per copy
  Csr Pb, Rb;               // n_b x n_cb prolongation of one copy, and its transpose
  Csr GK, GKt;              // FSAI of K = A_inn[F, F], embedded in n_b x n_b (fine rows and columns)
  double omegaK = 1.0;      // damping of the fine-point smoother
  std::vector<double> jdC;  // coarse rows: omega_C / a_ll (the FSAI of C-bar with a diagonal pattern); fine rows 0
  // A_c in the transformed basis (eq. "structAc" under P_s): block i is
  // Ac0 + the interface couplings of block i, Ac0 = P_b^T A_inn P_b; the
  // couplings are the fine ones (ivals, [entry][block]) at coarse indices
  Csr Ac0;
  std::vector<int32_t> cirow, cicol;
  std::vector<double> civals;
  // the full reduced operator A_c (n_cb * 2^s rows, copy index fastest) as
  // the finest level of its own AMG hierarchy (and device copies)
  std::shared_ptr<amgsym_problem> coarse;
};

}  // namespace amgsym

struct amgsym_problem {
  int64_t n = 0;      // full unknowns
  int64_t n_b = 0;    // base-block rows, n / 2^s
  int32_t s = 0;
  int32_t nb = 1;     // 2^s
  amgsym::Csr Ainn;   // H_0, columns sorted (AMGR's coarse problem: the shape only; its
                      // matrix is the finest level of its hierarchy)
  // Interface couplings: entries sorted by (row, col); ivals[e * nb + i] =
  // (A_out,i)[row, col].
  std::vector<int32_t> irow, icol;
  std::vector<double> ivals;
  std::vector<int32_t> perm;  // [nb][n_b]
  bool singular = false;      // every row sums to zero (pure Neumann): A 1 = 0
  // the full operator's CSR pattern (natural order), kept for
  // amgsym_update_values: 8 bytes per row + 4 per stored entry
  std::vector<int64_t> full_ptr;
  std::vector<int32_t> full_idx;
  amgsym_opts opts{};
  bool have_hierarchy = false;
  amgsym::HostHierarchy H;
  std::shared_ptr<amgsym::HostAmgr> amgr;  // AMGR top level (opts.amgr)
  amgsym::Device* dev = nullptr;
};

namespace amgsym {
// host_amg.cpp
// the hierarchy of A (taken by value: pass an rvalue to hand the matrix over)
void build_hierarchy(Csr A, const amgsym_opts& o, HostHierarchy& H);
// classical strength: strong[e] = 1 when -a_ij >= theta max_k (-a_ik) (entry e = (i, j))
std::vector<uint8_t> strength(const Csr& A, double theta);
// extended+i interpolation for the splitting cf (1 = C, -1 = F), truncated
Csr ext_i_interp(const Csr& A, const std::vector<uint8_t>& strong, const std::vector<int8_t>& cf, double trunc,
                 int max_elems);
// static FSAI factor G (G^T G ~ A^{-1}) on the strongest lower pattern
Csr fsai(const Csr& A, int max_lower);
// power-iteration estimate of lambda_max(G A G^T)
double lambda_max_GAGt(const Csr& A, const Csr& G, const Csr& Gt, uint64_t seed);
// host_amgr.cpp
void build_amgr(amgsym_problem* p, const amgsym_opts& o);
Csr transpose(const Csr& A);
// the entries e with keep[e] != 0, unit values
Csr pattern_of(const Csr& A, const std::vector<uint8_t>& keep);
Csr spgemm(const Csr& A, const Csr& B);
void sort_rows(Csr& A);
// solve.cu
void device_upload(amgsym_problem* p);
void device_free(amgsym_problem* p);
}  // namespace amgsym
