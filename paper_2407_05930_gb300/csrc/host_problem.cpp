// Problem creation, validation and extraction of the symmetry blocks (host),
// plus the structured-grid finite-volume generator.
//
// Sec. 2 of the paper: with the mirrored ordering (eq. "fields_struct") the
// operator has the dyadic block structure of eq. "struct_2sym", block (p, q)
// = H_{p XOR q}, and only H_0 (= H_inn of eq. "split_s") and the very sparse
// outer couplings H_m, m >= 1, need to be stored (memory / 2^s).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>

#include "internal.h"

namespace amgsym {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(amgsym_status code, const std::string& msg) { throw Error{code, msg}; }

}  // namespace amgsym

using namespace amgsym;

#define API_BEGIN try {
#define API_END                                                  \
  }                                                              \
  catch (const amgsym::Error& e) {                               \
    amgsym::set_last_error(e.msg);                               \
    return e.code;                                               \
  }                                                              \
  catch (const std::bad_alloc&) {                                \
    amgsym::set_last_error("host allocation failed");            \
    return AMGSYM_ERR_OOM;                                       \
  }                                                              \
  catch (...) {                                                  \
    amgsym::set_last_error("unexpected internal error");         \
    return AMGSYM_ERR_ARG;                                       \
  }                                                              \
  return AMGSYM_OK;

extern "C" const char* amgsym_last_error(void) { return amgsym::g_last_error.c_str(); }

extern "C" void amgsym_opts_default(amgsym_opts* o) {
  if (!o) return;
  o->strength_theta = 0.25;
  o->interp_trunc = 0.2;
  o->interp_max_elems = 3;
  o->max_levels = 25;
  o->coarse_max = 256;
  o->fsai_max_lower = 4;
  o->omega_scale = 1.2;
  o->nu = 1;
  o->precisions = 3;
  o->host_only = 0;
  o->seed = 12345;
  o->coarse_drop = 0.003;
  o->dia_max_diag = AMGSYM_MAX_DIAG;
  o->fuse_rows = 0;
  o->fsai_max_lower_coarse = 1;
  o->halo_kb = 0;
  o->amgr = 0;
  o->amgr_distance = 1;
  o->amgr_interp_max = 4;
  o->amgr_sym_ac = 1;
  o->zmarch = 0;
  o->sell = 0;
  o->lambda_device = 1;
}

extern "C" void amgsym_solve_opts_default(amgsym_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->maxit = 500;
  o->precision = AMGSYM_PREC_FP64;
  o->use_x0 = 0;
  o->inner_tol = 3e-7;
  o->max_outer = 20;
  o->finest_hat = 0;
  o->use_graph = 1;
  o->preconditioner = AMGSYM_PC_AMG;
  o->tune = 0;
}

// Sign of entry (i, j) of the Sylvester-Hadamard matrix 2^{s/2} P_s (eq. "P_s").
static inline double hsign(int i, int j) { return (__builtin_popcount((unsigned)(i & j)) & 1) ? -1.0 : 1.0; }

// The blocks of a full operator in mirrored order (Sec. 2): A_inn = H_0 and
// the interface couplings A_out,i, after validating the CSR, the map, the
// block structure of eq. "struct_2sym", symmetry and the diagonal.  Throws
// (through fail) on any violation; nothing is modified then.
struct Blocks {
  Csr Ainn;
  std::vector<int32_t> irow, icol;
  std::vector<double> ivals;
  bool singular = false;  // every row sums to zero: the constant spans the null space
};

static Blocks extract_blocks(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                             int32_t s, const int32_t* perm) {
  const int32_t nb = 1 << s;
  const int64_t n_b = n / nb;
  // CSR sanity.
  if (rowptr[0] != 0) fail(AMGSYM_ERR_ARG, "rowptr[0] != 0");
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) fail(AMGSYM_ERR_ARG, "rowptr not monotone");
  const int64_t nnz = rowptr[n];
  for (int64_t e = 0; e < nnz; ++e)
    if (colidx[e] < 0 || colidx[e] >= n) fail(AMGSYM_ERR_ARG, "column index out of range");
  // Map: bijection, inverse (copy, local index) of every natural index.
  std::vector<int32_t> copy_of(n, -1), local_of(n, -1);
  for (int32_t j = 0; j < nb; ++j)
    for (int64_t l = 0; l < n_b; ++l) {
      const int64_t p = perm[j * n_b + l];
      if (p < 0 || p >= n) fail(AMGSYM_ERR_MAP, "perm entry out of range");
      if (copy_of[p] >= 0) fail(AMGSYM_ERR_MAP, "perm is not a bijection (repeated index)");
      copy_of[p] = j;
      local_of[p] = (int32_t)l;
    }
  // Blocks H_m from the rows of copy 0 (eq. "struct_2sym": row block 0 holds
  // H_0 ... H_{2^s-1}).
  std::vector<Csr> Hm(nb);
  for (int32_t m = 0; m < nb; ++m) {
    Hm[m].rows = Hm[m].cols = n_b;
    Hm[m].ptr.assign(n_b + 1, 0);
  }
  for (int64_t l = 0; l < n_b; ++l) {
    const int64_t p = perm[l];
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) Hm[copy_of[colidx[e]]].ptr[l + 1]++;
  }
  for (int32_t m = 0; m < nb; ++m) {
    for (int64_t l = 0; l < n_b; ++l) Hm[m].ptr[l + 1] += Hm[m].ptr[l];
    Hm[m].idx.resize(Hm[m].ptr[n_b]);
    Hm[m].val.resize(Hm[m].ptr[n_b]);
  }
  {
    std::vector<std::vector<int64_t>> fill(nb);
    for (int32_t m = 0; m < nb; ++m) fill[m].assign(Hm[m].ptr.begin(), Hm[m].ptr.end() - 1);
    for (int64_t l = 0; l < n_b; ++l) {
      const int64_t p = perm[l];
      for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
        const int32_t q = colidx[e];
        const int32_t m = copy_of[q];
        const int64_t k = fill[m][l]++;
        Hm[m].idx[k] = local_of[q];
        Hm[m].val[k] = vals[e];
      }
    }
  }
  for (int32_t m = 0; m < nb; ++m) {
    sort_rows(Hm[m]);
    // duplicates are not allowed
    for (int64_t l = 0; l < n_b; ++l)
      for (int64_t e = Hm[m].ptr[l] + 1; e < Hm[m].ptr[l + 1]; ++e)
        if (Hm[m].idx[e] == Hm[m].idx[e - 1]) fail(AMGSYM_ERR_ARG, "duplicate entry in a CSR row");
  }
  // Validation: every stored entry matches its block, and no block entry is
  // missing from any row (counts agree).
  auto lookup = [&](const Csr& M, int64_t r, int32_t c, double* v) -> bool {
    const int32_t* b = M.idx.data() + M.ptr[r];
    const int32_t* e = M.idx.data() + M.ptr[r + 1];
    const int32_t* it = std::lower_bound(b, e, c);
    if (it == e || *it != c) return false;
    *v = M.val[it - M.idx.data()];
    return true;
  };
  for (int64_t p = 0; p < n; ++p) {
    const int32_t J = copy_of[p];
    const int32_t l = local_of[p];
    int64_t expect = 0;
    for (int32_t m = 0; m < nb; ++m) expect += Hm[m].ptr[l + 1] - Hm[m].ptr[l];
    if (rowptr[p + 1] - rowptr[p] != expect)
      fail(AMGSYM_ERR_NOT_SYMMETRIC, "row " + std::to_string(p) +
                                         " does not repeat the pattern of its base row (eq. struct_2sym)");
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      const int32_t q = colidx[e];
      const int32_t m = J ^ copy_of[q];
      double v;
      if (!lookup(Hm[m], l, local_of[q], &v) || v != vals[e])
        fail(AMGSYM_ERR_NOT_SYMMETRIC, "entry (" + std::to_string(p) + ", " + std::to_string(q) +
                                           ") differs from block H_" + std::to_string(m) +
                                           " (eq. struct_2sym)");
    }
  }
  // Symmetry of A <=> every H_m symmetric.
  for (int32_t m = 0; m < nb; ++m)
    for (int64_t l = 0; l < n_b; ++l)
      for (int64_t e = Hm[m].ptr[l]; e < Hm[m].ptr[l + 1]; ++e) {
        double v;
        if (!lookup(Hm[m], Hm[m].idx[e], (int32_t)l, &v) || v != Hm[m].val[e])
          fail(AMGSYM_ERR_NOT_SYMMETRIC, "matrix is not symmetric");
      }
  for (int64_t l = 0; l < n_b; ++l) {
    double v;
    if (!lookup(Hm[0], l, (int32_t)l, &v) || !(v > 0.0))
      fail(AMGSYM_ERR_NOT_SPD, "non-positive or missing diagonal entry");
  }

  Blocks B;
  // Pure Neumann (the paper's model problem, Sec. 2.2): every row sums to
  // zero up to rounding, so A 1 = 0 and the system is singular.
  B.singular = true;
  for (int64_t p = 0; p < n && B.singular; ++p) {
    double sum = 0.0, diag = 0.0, mag = 0.0;
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      sum += vals[e];
      mag += std::fabs(vals[e]);
      if (colidx[e] == p) diag = vals[e];
    }
    if (!(std::fabs(sum) <= 1e-12 * mag) || !(diag > 0.0)) B.singular = false;
  }
  // Interface couplings A_out,i = sum_{m>=1} sign(i, m) H_m (eq. "hL_splitting").
  for (int64_t l = 0; l < n_b; ++l) {
    std::vector<int32_t> cols;
    for (int32_t m = 1; m < nb; ++m)
      for (int64_t e = Hm[m].ptr[l]; e < Hm[m].ptr[l + 1]; ++e) cols.push_back(Hm[m].idx[e]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    for (int32_t c : cols) {
      B.irow.push_back((int32_t)l);
      B.icol.push_back(c);
      for (int32_t i = 0; i < nb; ++i) {
        double acc = 0.0;
        for (int32_t m = 1; m < nb; ++m) {
          double v;
          if (lookup(Hm[m], l, c, &v)) acc += hsign(i, m) * v;
        }
        B.ivals.push_back(acc);
      }
    }
  }
  B.Ainn = std::move(Hm[0]);
  return B;
}

extern "C" amgsym_status amgsym_create_problem(int64_t n, const int64_t* rowptr,
                                               const int32_t* colidx, const double* vals,
                                               int32_t s, const int32_t* perm, amgsym_t* out) {
  API_BEGIN
  if (!out) fail(AMGSYM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!rowptr || !colidx || !vals || !perm) fail(AMGSYM_ERR_ARG, "NULL input array");
  if (n <= 0) fail(AMGSYM_ERR_ARG, "n must be positive");
  if (s < 0 || s > 10) fail(AMGSYM_ERR_ARG, "s out of range [0, 10]");
  const int32_t nb = 1 << s;
  if (n % nb) fail(AMGSYM_ERR_MAP, "n is not divisible by 2^s");
  if (n / nb > INT32_MAX - 1) fail(AMGSYM_ERR_ARG, "base block too large for 32-bit indices");
  Blocks B = extract_blocks(n, rowptr, colidx, vals, s, perm);
  auto* P = new amgsym_problem();
  std::unique_ptr<amgsym_problem> guard(P);
  P->n = n;
  P->n_b = n / nb;
  P->s = s;
  P->nb = nb;
  P->Ainn = std::move(B.Ainn);
  P->irow = std::move(B.irow);
  P->icol = std::move(B.icol);
  P->ivals = std::move(B.ivals);
  P->singular = B.singular;
  P->perm.assign(perm, perm + n);
  // the pattern, for amgsym_update_values
  P->full_ptr.assign(rowptr, rowptr + n + 1);
  P->full_idx.assign(colidx, colidx + rowptr[n]);
  amgsym_opts_default(&P->opts);
  *out = guard.release();
  API_END
}

extern "C" amgsym_status amgsym_update_values(amgsym_t h, const double* vals) {
  API_BEGIN
  if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
  if (!vals) fail(AMGSYM_ERR_ARG, "NULL vals");
  // validate and extract first: a rejected update leaves the problem as it was
  Blocks B = extract_blocks(h->n, h->full_ptr.data(), h->full_idx.data(), vals, h->s, h->perm.data());
  device_free(h);
  h->have_hierarchy = false;
  h->H = HostHierarchy();
  h->amgr.reset();
  h->Ainn = std::move(B.Ainn);
  h->irow = std::move(B.irow);
  h->icol = std::move(B.icol);
  h->ivals = std::move(B.ivals);
  h->singular = B.singular;
  API_END
}

extern "C" int32_t amgsym_is_singular(amgsym_t h) { return h ? (h->singular ? 1 : 0) : -1; }

extern "C" amgsym_status amgsym_problem_sizes(amgsym_t h, int64_t* n, int64_t* n_b, int32_t* s,
                                              int64_t* nnz_inn, int64_t* n_iface_rows,
                                              int64_t* n_iface_entries) {
  API_BEGIN
  if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
  if (n) *n = h->n;
  if (n_b) *n_b = h->n_b;
  if (s) *s = h->s;
  if (nnz_inn) *nnz_inn = h->Ainn.nnz();
  if (n_iface_rows) {
    int64_t c = 0;
    for (size_t e = 0; e < h->irow.size(); ++e)
      if (e == 0 || h->irow[e] != h->irow[e - 1]) ++c;
    *n_iface_rows = c;
  }
  if (n_iface_entries) *n_iface_entries = (int64_t)h->irow.size();
  API_END
}

extern "C" amgsym_status amgsym_get_inner_block(amgsym_t h, int64_t* rowptr, int32_t* colidx,
                                                double* vals) {
  API_BEGIN
  if (!h || !rowptr || !colidx || !vals) fail(AMGSYM_ERR_ARG, "NULL argument");
  std::memcpy(rowptr, h->Ainn.ptr.data(), sizeof(int64_t) * h->Ainn.ptr.size());
  std::memcpy(colidx, h->Ainn.idx.data(), sizeof(int32_t) * h->Ainn.idx.size());
  std::memcpy(vals, h->Ainn.val.data(), sizeof(double) * h->Ainn.val.size());
  API_END
}

extern "C" amgsym_status amgsym_get_interface(amgsym_t h, int32_t* row, int32_t* col, double* vals) {
  API_BEGIN
  if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
  if (h->irow.empty()) return AMGSYM_OK;
  if (!row || !col || !vals) fail(AMGSYM_ERR_ARG, "NULL argument");
  std::memcpy(row, h->irow.data(), sizeof(int32_t) * h->irow.size());
  std::memcpy(col, h->icol.data(), sizeof(int32_t) * h->icol.size());
  std::memcpy(vals, h->ivals.data(), sizeof(double) * h->ivals.size());
  API_END
}

extern "C" void amgsym_destroy(amgsym_t h) {
  if (!h) return;
  try {
    device_free(h);
  } catch (...) {
  }
  delete h;
}

// --------------------------------------------------------------------------
// Structured-grid generator.

extern "C" amgsym_status amgsym_grid_widths(int64_t N, double gamma, double* w) {
  API_BEGIN
  if (N <= 0 || !w) fail(AMGSYM_ERR_ARG, "bad arguments");
  std::vector<double> x(N + 1);
  for (int64_t i = 0; i <= N; ++i) {
    if (gamma == 0.0)
      x[i] = (double)i / (double)N;
    else
      x[i] = 0.5 * (1.0 + std::tanh(gamma * (2.0 * (double)i / (double)N - 1.0)) / std::tanh(gamma));
  }
  x[0] = 0.0;
  x[N] = 1.0;
  for (int64_t i = 0; i < N; ++i) w[i] = x[i + 1] - x[i];
  if (N % 2 == 0)
    for (int64_t i = 0; i < N / 2; ++i) w[N - 1 - i] = w[i];
  API_END
}

static void check_grid(int32_t d, const int64_t* N) {
  if (d < 1 || d > 3 || !N) fail(AMGSYM_ERR_ARG, "grid dimension must be 1..3");
  for (int a = 0; a < d; ++a)
    if (N[a] <= 0) fail(AMGSYM_ERR_ARG, "grid extent must be positive");
}

extern "C" int64_t amgsym_fv_nnz(int32_t d, const int64_t* N) {
  if (d < 1 || d > 3 || !N) return -1;
  int64_t n = 1;
  for (int a = 0; a < d; ++a) n *= N[a];
  int64_t nnz = n;
  for (int a = 0; a < d; ++a) nnz += 2 * (n / N[a]) * (N[a] - 1);
  return nnz;
}

extern "C" amgsym_status amgsym_fv_assemble(int32_t d, const int64_t* N, const double* widths,
                                            const double* k, int64_t* rowptr, int32_t* colidx,
                                            double* vals) {
  return amgsym_fv_assemble_bc(d, N, widths, k, AMGSYM_BC_DIRICHLET, rowptr, colidx, vals);
}

extern "C" amgsym_status amgsym_fv_assemble_bc(int32_t d, const int64_t* N, const double* widths,
                                               const double* k, int32_t bc, int64_t* rowptr,
                                               int32_t* colidx, double* vals) {
  API_BEGIN
  check_grid(d, N);
  if (bc != AMGSYM_BC_DIRICHLET && bc != AMGSYM_BC_NEUMANN) fail(AMGSYM_ERR_ARG, "unknown boundary condition");
  // a wall face carries the Dirichlet transmissibility, or no flux (Neumann)
  const double wall = bc == AMGSYM_BC_NEUMANN ? 0.0 : 1.0;
  if (!widths || !k || !rowptr || !colidx || !vals) fail(AMGSYM_ERR_ARG, "NULL argument");
  int64_t E[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) E[a] = N[a];
  const int64_t n = E[0] * E[1] * E[2];
  if (n > INT32_MAX) fail(AMGSYM_ERR_ARG, "grid too large for 32-bit column indices");
  const double* h[3];
  static const double one = 1.0;
  int64_t off = 0;
  for (int a = 0; a < 3; ++a) {
    if (a < d) {
      h[a] = widths + off;
      off += N[a];
    } else {
      h[a] = &one;
    }
  }
  const int64_t stride[3] = {1, E[0], E[0] * E[1]};
  auto hw = [&](int a, int64_t i) { return a < d ? h[a][i] : 1.0; };
  // Row p = (i0, i1, i2); neighbours in increasing column order:
  // -z, -y, -x, self, +x, +y, +z.
  int64_t pos = 0;
  rowptr[0] = 0;
  for (int64_t i2 = 0; i2 < E[2]; ++i2)
    for (int64_t i1 = 0; i1 < E[1]; ++i1)
      for (int64_t i0 = 0; i0 < E[0]; ++i0) {
        const int64_t c[3] = {i0, i1, i2};
        const int64_t p = i0 + E[0] * (i1 + E[1] * i2);
        double tlo[3] = {0, 0, 0}, thi[3] = {0, 0, 0};
        bool has_lo[3] = {false, false, false}, has_hi[3] = {false, false, false};
        for (int a = 0; a < d; ++a) {
          double area = 1.0;
          for (int b = 0; b < d; ++b)
            if (b != a) area *= hw(b, c[b]);
          const double rp = hw(a, c[a]) / (2.0 * k[p]);
          // low face
          if (c[a] > 0) {
            const int64_t q = p - stride[a];
            const double rq = hw(a, c[a] - 1) / (2.0 * k[q]);
            tlo[a] = area / (rq + rp);
            has_lo[a] = true;
          } else {
            tlo[a] = wall * (area / rp);
          }
          if (c[a] < E[a] - 1) {
            const int64_t q = p + stride[a];
            const double rq = hw(a, c[a] + 1) / (2.0 * k[q]);
            thi[a] = area / (rp + rq);
            has_hi[a] = true;
          } else {
            thi[a] = wall * (area / rp);
          }
        }
        double diag = 0.0;
        for (int a = 0; a < d; ++a) diag += (tlo[a] + thi[a]);
        for (int a = d - 1; a >= 0; --a)
          if (has_lo[a]) {
            colidx[pos] = (int32_t)(p - stride[a]);
            vals[pos++] = -tlo[a];
          }
        colidx[pos] = (int32_t)p;
        vals[pos++] = diag;
        for (int a = 0; a < d; ++a)
          if (has_hi[a]) {
            colidx[pos] = (int32_t)(p + stride[a]);
            vals[pos++] = -thi[a];
          }
        rowptr[p + 1] = pos;
      }
  API_END
}

extern "C" amgsym_status amgsym_mirror_perm(int32_t d, const int64_t* N, int32_t s, int32_t* perm) {
  API_BEGIN
  check_grid(d, N);
  if (!perm) fail(AMGSYM_ERR_ARG, "NULL perm");
  if (s < 0 || s > d) fail(AMGSYM_ERR_ARG, "s must be in [0, d]");
  int64_t E[3] = {1, 1, 1}, M[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) E[a] = M[a] = N[a];
  for (int b = 0; b < s; ++b) {
    if (N[b] % 2) fail(AMGSYM_ERR_ARG, "a mirrored axis needs an even number of cells");
    M[b] = N[b] / 2;
  }
  const int64_t n_b = M[0] * M[1] * M[2];
  if (E[0] * E[1] * E[2] > INT32_MAX) fail(AMGSYM_ERR_ARG, "grid too large for int32 map");
  for (int32_t j = 0; j < (1 << s); ++j) {
    int64_t l = 0;
    for (int64_t i2 = 0; i2 < M[2]; ++i2)
      for (int64_t i1 = 0; i1 < M[1]; ++i1)
        for (int64_t i0 = 0; i0 < M[0]; ++i0, ++l) {
          int64_t c[3] = {i0, i1, i2};
          for (int b = 0; b < s; ++b)
            if ((j >> b) & 1) c[b] = E[b] - 1 - c[b];
          perm[j * n_b + l] = (int32_t)(c[0] + E[0] * (c[1] + E[1] * c[2]));
        }
  }
  API_END
}
