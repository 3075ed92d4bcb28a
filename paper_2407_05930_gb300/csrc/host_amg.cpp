// Host setup of the AMG hierarchy of A_inn (Sec. 2.2 eq. "AMGinn"; Sec. 5).
//
// The paper's AMG for this path: classical (C/F) coarsening by PMIS
// (De Sterck, Yang, Heys 2006), extended+i interpolation (De Sterck,
// Falgout, Nolting, Yang 2008), an FSAI smoother and a direct solve on the
// coarsest level.  The paper does not fix the strength threshold, the
// interpolation truncation, the FSAI pattern, the damping or the coarse size;
// the defaults of amgsym_opts_default are this library's choices.
//
// Everything here runs once per setup; none of it is on the timed solve path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <random>
#include <string>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "internal.h"

namespace amgsym {

// Sorts the entries e in [b, e) of A by column, through the scratch tmp.
static void sort_range(Csr& A, int64_t b, int64_t e, std::vector<std::pair<int32_t, double>>& tmp) {
  tmp.resize(e - b);
  for (int64_t k = b; k < e; ++k) tmp[k - b] = {A.idx[k], A.val[k]};
  std::sort(tmp.begin(), tmp.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  for (int64_t k = b; k < e; ++k) {
    A.idx[k] = tmp[k - b].first;
    A.val[k] = tmp[k - b].second;
  }
}

void sort_rows(Csr& A) {
#pragma omp parallel
  {
    std::vector<std::pair<int32_t, double>> tmp;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i = 0; i < A.rows; ++i) {
      const int64_t b = A.ptr[i], e = A.ptr[i + 1];
      bool sorted = true;
      for (int64_t k = b + 1; k < e; ++k)
        if (A.idx[k] < A.idx[k - 1]) {
          sorted = false;
          break;
        }
      if (!sorted) sort_range(A, b, e, tmp);
    }
  }
}

static int host_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Rows of T = A^T come out in ascending source-row order.  Large matrices
// are split into contiguous chunks of source rows: each chunk counts its
// entries per column, a column's slots are handed out chunk after chunk,
// and each chunk fills its slots in row order, which gives the same arrays
// as one sequential pass.
Csr transpose(const Csr& A) {
  Csr T;
  T.rows = A.cols;
  T.cols = A.rows;
  T.ptr.assign(T.rows + 1, 0);
  const int64_t nnz = A.nnz();
  T.idx.resize(nnz);
  T.val.resize(nnz);
  // chunks: one per thread (at most 16), with the 4-byte column counters of
  // all chunks at most half the 12 bytes per entry of the matrix
  int64_t nch = nnz < (int64_t)1 << 20 ? 1 : std::min<int64_t>(std::min(host_threads(), 16), A.rows);
  nch = std::min<int64_t>(nch, std::max<int64_t>(1, 3 * nnz / (2 * std::max<int64_t>(A.cols, 1))));
  if (nch <= 1) {
    for (int64_t e = 0; e < nnz; ++e) T.ptr[A.idx[e] + 1]++;
    for (int64_t i = 0; i < T.rows; ++i) T.ptr[i + 1] += T.ptr[i];
    std::vector<int64_t> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t i = 0; i < A.rows; ++i)
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int64_t k = fill[A.idx[e]]++;
        T.idx[k] = (int32_t)i;
        T.val[k] = A.val[e];
      }
    return T;
  }
  const int64_t nc = T.rows;
  // cnt[k * nc + c]: entries of chunk k in column c, then that chunk's first
  // slot within the column (a column holds < 2^31 entries: int32 indices)
  std::unique_ptr<int32_t[]> cnt(new int32_t[(size_t)(nch * nc)]);
  auto row0 = [&](int64_t k) { return A.rows * k / nch; };
#pragma omp parallel for schedule(static, 1)
  for (int64_t k = 0; k < nch; ++k) {
    int32_t* ck = cnt.get() + k * nc;
    std::fill(ck, ck + nc, 0);
    for (int64_t e = A.ptr[row0(k)]; e < A.ptr[row0(k + 1)]; ++e) ck[A.idx[e]]++;
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    int32_t run = 0;
    for (int64_t k = 0; k < nch; ++k) {
      const int32_t v = cnt[k * nc + c];
      cnt[k * nc + c] = run;
      run += v;
    }
    T.ptr[c + 1] = run;
  }
  for (int64_t c = 0; c < nc; ++c) T.ptr[c + 1] += T.ptr[c];
#pragma omp parallel for schedule(static, 1)
  for (int64_t k = 0; k < nch; ++k) {
    int32_t* ck = cnt.get() + k * nc;
    for (int64_t i = row0(k); i < row0(k + 1); ++i)
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int32_t c = A.idx[e];
        const int64_t slot = T.ptr[c] + ck[c]++;
        T.idx[slot] = (int32_t)i;
        T.val[slot] = A.val[e];
      }
  }
  return T;
}

// The entries e of A with keep[e] set, as a pattern (unit values), rows in
// A's order.
Csr pattern_of(const Csr& A, const std::vector<uint8_t>& keep) {
  const int64_t n = A.rows;
  Csr S;
  S.rows = n;
  S.cols = A.cols;
  S.ptr.assign(n + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) c += keep[e] != 0;
    S.ptr[i + 1] = c;
  }
  for (int64_t i = 0; i < n; ++i) S.ptr[i + 1] += S.ptr[i];
  S.idx.resize(S.ptr[n]);
  S.val.assign(S.ptr[n], 1.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t w = S.ptr[i];
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
      if (keep[e]) S.idx[w++] = A.idx[e];
  }
  return S;
}

// C = A B (Gustavson, two passes, rows sorted, exact zeros kept out only if
// both operands had no entry there).
Csr spgemm(const Csr& A, const Csr& B) {
  Csr C;
  C.rows = A.rows;
  C.cols = B.cols;
  C.ptr.assign(C.rows + 1, 0);
#pragma omp parallel
  {
    std::vector<int64_t> mark(B.cols, -1);
#pragma omp for schedule(dynamic, 512)
    for (int64_t i = 0; i < A.rows; ++i) {
      int64_t cnt = 0;
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int32_t k = A.idx[e];
        for (int64_t f = B.ptr[k]; f < B.ptr[k + 1]; ++f) {
          const int32_t j = B.idx[f];
          if (mark[j] != i) {
            mark[j] = i;
            ++cnt;
          }
        }
      }
      C.ptr[i + 1] = cnt;
    }
  }
  for (int64_t i = 0; i < C.rows; ++i) C.ptr[i + 1] += C.ptr[i];
  C.idx.resize(C.ptr[C.rows]);
  C.val.resize(C.ptr[C.rows]);
#pragma omp parallel
  {
    std::vector<int64_t> pos(B.cols, -1);
    std::vector<std::pair<int32_t, double>> tmp;
#pragma omp for schedule(dynamic, 512)
    for (int64_t i = 0; i < A.rows; ++i) {
      int64_t w = C.ptr[i];
      const int64_t start = w;
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int32_t k = A.idx[e];
        const double a = A.val[e];
        for (int64_t f = B.ptr[k]; f < B.ptr[k + 1]; ++f) {
          const int32_t j = B.idx[f];
          if (pos[j] < start) {
            pos[j] = w;
            C.idx[w] = j;
            C.val[w] = a * B.val[f];
            ++w;
          } else {
            C.val[pos[j]] += a * B.val[f];
          }
        }
      }
      sort_range(C, start, w, tmp);
    }
  }
  return C;
}

static void spmv(const Csr& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign(A.rows, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A.rows; ++i) {
    double acc = 0.0;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) acc += A.val[e] * x[A.idx[e]];
    y[i] = acc;
  }
}

static inline double find(const Csr& A, int64_t r, int32_t c) {
  const int32_t* b = A.idx.data() + A.ptr[r];
  const int32_t* e = A.idx.data() + A.ptr[r + 1];
  const int32_t* it = std::lower_bound(b, e, c);
  return (it != e && *it == c) ? A.val[it - A.idx.data()] : 0.0;
}

// Classical strength of connection: j in S_i iff -a_ij >= theta max_{k != i} (-a_ik).
std::vector<uint8_t> strength(const Csr& A, double theta) {
  std::vector<uint8_t> strong(A.nnz(), 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A.rows; ++i) {
    double mx = 0.0;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
      if (A.idx[e] != i) mx = std::max(mx, -A.val[e]);
    if (mx <= 0.0) continue;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
      if (A.idx[e] != i && -A.val[e] >= theta * mx) strong[e] = 1;
  }
  return strong;
}

// PMIS coarsening (De Sterck, Yang, Heys 2006): cf[i] = 1 (C) or -1 (F).
static std::vector<int8_t> pmis(const Csr& A, const std::vector<uint8_t>& strong, uint64_t seed) {
  const int64_t n = A.rows;
  // S: for each i, the j that i strongly depends on; S^T: the j that
  // strongly depend on i.
  Csr S = pattern_of(A, strong);
  Csr ST = transpose(S);
  std::vector<double> measure(n);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  for (int64_t i = 0; i < n; ++i) measure[i] = (double)(ST.ptr[i + 1] - ST.ptr[i]) + U(rng);
  std::vector<int8_t> cf(n, 0);
  int64_t undecided = 0;
#pragma omp parallel for schedule(static) reduction(+ : undecided)
  for (int64_t i = 0; i < n; ++i) {
    if (ST.ptr[i + 1] == ST.ptr[i]) cf[i] = -1;  // influences nobody
    else ++undecided;
  }
  std::vector<int8_t> newc(n, 0);
  int guard = 0;
  while (undecided > 0 && guard++ < 1000) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      newc[i] = 0;
      if (cf[i] != 0) continue;
      bool best = true;
      for (int64_t e = S.ptr[i]; e < S.ptr[i + 1] && best; ++e) {
        const int32_t j = S.idx[e];
        if (cf[j] == 0 && measure[j] >= measure[i]) best = false;
      }
      for (int64_t e = ST.ptr[i]; e < ST.ptr[i + 1] && best; ++e) {
        const int32_t j = ST.idx[e];
        if (cf[j] == 0 && measure[j] >= measure[i]) best = false;
      }
      newc[i] = best ? 1 : 0;
    }
    // the new C points; every other undecided point that strongly depends
    // on one of them (a new C point in its row of S) becomes F
    undecided = 0;
#pragma omp parallel for schedule(static) reduction(+ : undecided)
    for (int64_t i = 0; i < n; ++i) {
      if (cf[i] != 0) continue;
      if (newc[i]) {
        cf[i] = 1;
        continue;
      }
      bool f = false;
      for (int64_t e = S.ptr[i]; e < S.ptr[i + 1] && !f; ++e) f = newc[S.idx[e]] != 0;
      if (f) cf[i] = -1;
      else ++undecided;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    if (cf[i] == 0) cf[i] = 1;
  return cf;
}

// CSR from per-row lists of (column, value), in list order; the lists are
// released as they are copied.
static Csr from_rows(int64_t cols, std::vector<std::vector<std::pair<int32_t, double>>>& rows) {
  const int64_t n = (int64_t)rows.size();
  Csr M;
  M.rows = n;
  M.cols = cols;
  M.ptr.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) M.ptr[i + 1] = M.ptr[i] + (int64_t)rows[i].size();
  M.idx.resize(M.ptr[n]);
  M.val.resize(M.ptr[n]);
#pragma omp parallel for schedule(static, 4096)
  for (int64_t i = 0; i < n; ++i) {
    int64_t w = M.ptr[i];
    for (const auto& p : rows[i]) {
      M.idx[w] = p.first;
      M.val[w++] = p.second;
    }
    std::vector<std::pair<int32_t, double>>().swap(rows[i]);
  }
  return M;
}

// Extended+i interpolation (De Sterck, Falgout, Nolting, Yang 2008) with
// truncation to the `max_elems` largest weights above trunc * max, rescaled
// to keep the row sum.
Csr ext_i_interp(const Csr& A, const std::vector<uint8_t>& strong,
                        const std::vector<int8_t>& cf, double trunc, int max_elems) {
  const int64_t n = A.rows;
  std::vector<int32_t> cmap(n, -1);
  int32_t nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (cf[i] > 0) cmap[i] = nc++;
  std::vector<double> diag(n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) diag[i] = find(A, i, (int32_t)i);
  std::vector<std::vector<std::pair<int32_t, double>>> rows(n);
#pragma omp parallel
  {
    std::vector<int64_t> mark(n, -1);  // mark[j] == i  <=> j in C^_i
    std::vector<double> num(n, 0.0);
    std::vector<int32_t> chat;
    std::vector<std::pair<int32_t, double>> w;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      auto& out = rows[i];
      if (cf[i] > 0) {
        out.push_back({cmap[i], 1.0});
        continue;
      }
      chat.clear();
      // C^_i = strong C neighbours of i and of its strong F neighbours.
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        if (!strong[e]) continue;
        const int32_t j = A.idx[e];
        if (cf[j] > 0) {
          if (mark[j] != i) {
            mark[j] = i;
            chat.push_back(j);
          }
        } else {
          for (int64_t f = A.ptr[j]; f < A.ptr[j + 1]; ++f) {
            const int32_t l = A.idx[f];
            if (strong[f] && cf[l] > 0 && mark[l] != i) {
              mark[l] = i;
              chat.push_back(l);
            }
          }
        }
      }
      if (chat.empty()) continue;  // no interpolation: the smoother handles the point
      for (int32_t j : chat) num[j] = 0.0;
      double dt = 0.0;  // a~_ii
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int32_t j = A.idx[e];
        const double a = A.val[e];
        if (j == i) {
          dt += a;
        } else if (mark[j] == i) {
          num[j] += a;  // direct connection into C^_i (strong or weak)
        } else if (strong[e] && cf[j] < 0) {
          // strong F neighbour k = j: distribute over C^_i and i by a-bar
          const double akk = diag[j];
          double D = 0.0;
          for (int64_t f = A.ptr[j]; f < A.ptr[j + 1]; ++f) {
            const int32_t l = A.idx[f];
            const double v = A.val[f];
            if ((l == i || mark[l] == i) && l != j && (v * akk < 0.0)) D += v;
          }
          if (D == 0.0) {
            dt += a;
            continue;
          }
          for (int64_t f = A.ptr[j]; f < A.ptr[j + 1]; ++f) {
            const int32_t l = A.idx[f];
            const double v = A.val[f];
            if (l == j || !(v * akk < 0.0)) continue;
            if (l == i)
              dt += a * v / D;
            else if (mark[l] == i)
              num[l] += a * v / D;
          }
        } else {
          dt += a;  // weak connection outside C^_i: lumped to the diagonal
        }
      }
      if (dt == 0.0) continue;
      w.clear();
      double sum_all = 0.0;
      for (int32_t j : chat) {
        const double wij = -num[j] / dt;
        if (wij != 0.0) {
          w.push_back({j, wij});
          sum_all += wij;
        }
      }
      // truncation
      std::sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return std::fabs(x.second) > std::fabs(y.second); });
      double mx = w.empty() ? 0.0 : std::fabs(w[0].second);
      size_t keep = 0;
      while (keep < w.size() && (int)keep < max_elems && std::fabs(w[keep].second) >= trunc * mx) ++keep;
      w.resize(keep);
      double sum_keep = 0.0;
      for (auto& p : w) sum_keep += p.second;
      const double scale = (sum_keep != 0.0) ? sum_all / sum_keep : 1.0;
      for (auto& p : w) out.push_back({cmap[p.first], p.second * scale});
      std::sort(out.begin(), out.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    }
  }
  return from_rows(nc, rows);
}

// Small dense Cholesky solve A y = rhs in place (m x m, row-major); false if
// A is not numerically SPD.
static bool chol_solve(std::vector<double>& A, std::vector<double>& y, int m) {
  for (int j = 0; j < m; ++j) {
    double d = A[j * m + j];
    for (int k = 0; k < j; ++k) d -= A[j * m + k] * A[j * m + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double v = A[i * m + j];
      for (int k = 0; k < j; ++k) v -= A[i * m + k] * A[j * m + k];
      A[i * m + j] = v / d;
    }
  }
  for (int i = 0; i < m; ++i) {
    double v = y[i];
    for (int k = 0; k < i; ++k) v -= A[i * m + k] * y[k];
    y[i] = v / A[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < m; ++k) v -= A[k * m + i] * y[k];
    y[i] = v / A[i * m + i];
  }
  return true;
}

// Static FSAI: G lower triangular on the pattern {i} U (the max_lower-1
// strongest lower entries of row i), rows scaled so diag(G A G^T) = 1
// (eq. "Ginn": G^T G ~ A^{-1}).
Csr fsai(const Csr& A, int max_lower) {
  const int64_t n = A.rows;
  std::vector<std::vector<std::pair<int32_t, double>>> rows(n);
#pragma omp parallel
  {
    std::vector<std::pair<double, int32_t>> cand;
    std::vector<int32_t> pat;
    std::vector<double> M, y;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
      cand.clear();
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
        if (A.idx[e] < i && A.val[e] != 0.0) cand.push_back({-std::fabs(A.val[e]), A.idx[e]});
      std::sort(cand.begin(), cand.end());
      pat.clear();
      for (size_t k = 0; k < cand.size() && (int)k < max_lower - 1; ++k) pat.push_back(cand[k].second);
      std::sort(pat.begin(), pat.end());
      pat.push_back((int32_t)i);
      const int m = (int)pat.size();
      M.assign(m * m, 0.0);
      for (int r = 0; r < m; ++r)
        for (int c = 0; c <= r; ++c) {
          const double v = find(A, pat[r], pat[c]);
          M[r * m + c] = v;
          M[c * m + r] = v;
        }
      y.assign(m, 0.0);
      y[m - 1] = 1.0;
      auto& out = rows[i];
      if (chol_solve(M, y, m) && y[m - 1] > 0.0) {
        const double sc = 1.0 / std::sqrt(y[m - 1]);
        for (int r = 0; r < m; ++r) out.push_back({pat[r], y[r] * sc});
      } else {
        const double d = find(A, i, (int32_t)i);
        out.push_back({(int32_t)i, d > 0.0 ? 1.0 / std::sqrt(d) : 0.0});
      }
    }
  }
  return from_rows(n, rows);
}

// Largest eigenvalue of G A G^T by power iteration (an estimate from below;
// the damping keeps a margin).
double lambda_max_GAGt(const Csr& A, const Csr& G, const Csr& Gt, uint64_t seed) {
  const int64_t n = A.rows;
  std::vector<double> v(n), t1, t2, t3;
  std::mt19937_64 rng(seed ^ 0x9e3779b97f4a7c15ULL);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (auto& x : v) x = U(rng);
  double lam = 0.0;
  for (int it = 0; it < 30; ++it) {
    double nv = 0.0;
    for (double x : v) nv += x * x;
    nv = std::sqrt(nv);
    if (nv == 0.0) break;
    for (auto& x : v) x /= nv;
    spmv(Gt, v, t1);
    spmv(A, t1, t2);
    spmv(G, t2, t3);
    double num = 0.0;
    for (int64_t i = 0; i < n; ++i) num += v[i] * t3[i];
    lam = num;
    v.swap(t3);
  }
  return lam;
}

// Dense inverse of the coarsest operator by Cholesky.  A singular one whose
// null space is the constant vector (every row sums to zero: the coarsest
// level of a pure Neumann problem, whose interpolation reproduces constants)
// gets the pseudo-inverse instead: with e = 1/sqrt(m) and a the mean
// diagonal, B = A + a e e^T is positive definite and B^{-1} = A^+ + e e^T / a.
static std::vector<double> dense_inverse(const Csr& A) {
  const int64_t m = A.rows;
  std::vector<double> M(m * m, 0.0);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) M[i * m + A.idx[e]] = A.val[e];
  bool singular = m > 1;
  double diag_mean = 0.0;
  for (int64_t i = 0; i < m && singular; ++i) {
    double sum = 0.0, mag = 0.0;
    for (int64_t j = 0; j < m; ++j) {
      sum += M[i * m + j];
      mag += std::fabs(M[i * m + j]);
    }
    if (!(std::fabs(sum) <= 1e-10 * mag)) singular = false;
    diag_mean += M[i * m + i];
  }
  const double shift = singular ? diag_mean / (double)m : 0.0;
  if (singular)
    for (int64_t i = 0; i < m * m; ++i) M[i] += shift / (double)m;
  // symmetrise (the Galerkin product is symmetric up to rounding)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < i; ++j) {
      const double v = 0.5 * (M[i * m + j] + M[j * m + i]);
      M[i * m + j] = M[j * m + i] = v;
    }
  // Cholesky
  for (int64_t j = 0; j < m; ++j) {
    double d = M[j * m + j];
    for (int64_t k = 0; k < j; ++k) d -= M[j * m + k] * M[j * m + k];
    if (!(d > 0.0)) fail(AMGSYM_ERR_NOT_SPD, "coarsest-level matrix is not positive definite");
    d = std::sqrt(d);
    M[j * m + j] = d;
    for (int64_t i = j + 1; i < m; ++i) {
      double v = M[i * m + j];
      for (int64_t k = 0; k < j; ++k) v -= M[i * m + k] * M[j * m + k];
      M[i * m + j] = v / d;
    }
  }
  // inverse column by column
  std::vector<double> inv(m * m, 0.0), y(m);
  for (int64_t c = 0; c < m; ++c) {
    for (int64_t i = 0; i < m; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int64_t k = 0; k < i; ++k) v -= M[i * m + k] * y[k];
      y[i] = v / M[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) {
      double v = y[i];
      for (int64_t k = i + 1; k < m; ++k) v -= M[k * m + i] * y[k];
      y[i] = v / M[i * m + i];
    }
    for (int64_t i = 0; i < m; ++i) inv[i * m + c] = y[i];
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < i; ++j) {
      const double v = 0.5 * (inv[i * m + j] + inv[j * m + i]);
      inv[i * m + j] = inv[j * m + i] = v;
    }
  if (singular)
    for (int64_t i = 0; i < m * m; ++i) inv[i] -= 1.0 / (shift * (double)m);
  return inv;
}

// Sparsified Galerkin operator: off-diagonal entries with |a_ij| <
// theta sqrt(a_ii a_jj) (a symmetric test) are removed and added to the
// diagonal of their row, which keeps row sums and symmetry.  Removing a
// negative coupling of a diagonally dominant M-matrix keeps it weakly
// diagonally dominant, so the operator stays positive definite.
static Csr sparsify(const Csr& A, double theta) {
  if (theta <= 0.0) return A;
  const int64_t n = A.rows;
  std::vector<double> diag(n, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) diag[i] = find(A, i, (int32_t)i);
  Csr B;
  B.rows = A.rows;
  B.cols = A.cols;
  B.ptr.assign(n + 1, 0);
  std::vector<double> lump(n, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t cnt = 0;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const int32_t j = A.idx[e];
      const double thr = theta * std::sqrt(std::fabs(diag[i] * diag[j]));
      if (j == i || std::fabs(A.val[e]) >= thr)
        ++cnt;
      else
        lump[i] += A.val[e];
    }
    B.ptr[i + 1] = cnt;
  }
  for (int64_t i = 0; i < n; ++i) B.ptr[i + 1] += B.ptr[i];
  B.idx.resize(B.ptr[n]);
  B.val.resize(B.ptr[n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t w = B.ptr[i];
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const int32_t j = A.idx[e];
      const double thr = theta * std::sqrt(std::fabs(diag[i] * diag[j]));
      if (j == i) {
        B.idx[w] = j;
        B.val[w++] = A.val[e] + lump[i];
      } else if (std::fabs(A.val[e]) >= thr) {
        B.idx[w] = j;
        B.val[w++] = A.val[e];
      }
    }
  }
  return B;
}

// (A + A^T) / 2 for a matrix with a symmetric pattern and sorted rows
// without repeated columns (the Galerkin product: symmetric up to rounding);
// unchanged otherwise.  Each pair (i, j), (j, i) with j < i gets the mean of
// its two values; a diagonal entry stays as it is.
static void symmetrize(Csr& A) {
  const int64_t n = A.rows;
  if (A.cols != n) return;
  // the position of (j, i), or -1
  auto mirror = [&](int64_t i, int32_t j) -> int64_t {
    const int32_t* b = A.idx.data() + A.ptr[j];
    const int32_t* f = A.idx.data() + A.ptr[j + 1];
    const int32_t* it = std::lower_bound(b, f, (int32_t)i);
    return (it != f && *it == i) ? it - A.idx.data() : -1;
  };
  int64_t missing = 0;
#pragma omp parallel for schedule(static) reduction(+ : missing)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) missing += mirror(i, A.idx[e]) < 0;
  if (missing) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1] && A.idx[e] < i; ++e) {
      const int64_t f = mirror(i, A.idx[e]);
      const double v = 0.5 * (A.val[e] + A.val[f]);
      A.val[e] = v;
      A.val[f] = v;
    }
}

static constexpr int64_t kDenseLimit = 4096;

void build_hierarchy(Csr A0, const amgsym_opts& o, HostHierarchy& H) {
  H.levels.clear();
  H.levels.emplace_back();
  H.levels[0].A = std::move(A0);
  sort_rows(H.levels[0].A);
  for (int lev = 0;; ++lev) {
    HostLevel& L = H.levels[lev];
    const int64_t n = L.A.rows;
    bool coarsest = (n <= o.coarse_max) || (lev + 1 >= o.max_levels);
    Csr P;
    if (!coarsest) {
      auto strong = strength(L.A, o.strength_theta);
      auto cf = pmis(L.A, strong, o.seed + (uint64_t)lev);
      P = ext_i_interp(L.A, strong, cf, o.interp_trunc, o.interp_max_elems);
      if (P.cols == 0 || P.cols >= (int64_t)(0.9 * (double)n)) coarsest = true;
    }
    if (coarsest) {
      if (n > kDenseLimit)
        fail(AMGSYM_ERR_ARG, "coarsening stalled above the dense coarse-solve limit (" +
                                 std::to_string(n) + " rows)");
      L.coarse_inv = dense_inverse(L.A);
      break;
    }
    L.G = fsai(L.A, lev == 0 ? o.fsai_max_lower : o.fsai_max_lower_coarse);
    L.Gt = transpose(L.G);
    if (o.lambda_device && !o.host_only) {
      // estimated on the device after the upload (device_upload), same steps
      L.lambda_max = 0.0;
      L.omega = 0.0;
    } else {
      L.lambda_max = lambda_max_GAGt(L.A, L.G, L.Gt, o.seed + 17 * (uint64_t)lev);
      L.omega = (L.lambda_max > 0.0) ? o.omega_scale / L.lambda_max : 1.0;
    }
    L.P = std::move(P);
    L.R = transpose(L.P);
    Csr AP = spgemm(L.A, L.P);
    Csr Ac = spgemm(L.R, AP);
    symmetrize(Ac);
    Ac = sparsify(Ac, o.coarse_drop);
    H.levels.emplace_back();
    H.levels[lev + 1].A = std::move(Ac);
  }
}

// Diagonal-offset form (see Dia): distinct column offsets counted with an
// early exit, padding bounded, then exact symmetry checked diagonal by
// diagonal so that a symmetric stencil stores only its lower half.
Dia build_dia(const Csr& M, int max_diag) {
  Dia D;
  const int64_t n = M.rows;
  if (max_diag <= 0 || n <= 0 || M.cols != n || n > INT32_MAX) return D;
  max_diag = std::min(max_diag, kMaxDiag);
  std::vector<int64_t> offs;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = M.ptr[i]; e < M.ptr[i + 1]; ++e) {
      const int64_t o = (int64_t)M.idx[e] - i;
      if (std::find(offs.begin(), offs.end(), o) == offs.end()) {
        if ((int)offs.size() == max_diag) return D;
        offs.push_back(o);
      }
    }
  if (offs.empty() || (double)offs.size() * (double)n > 1.25 * (double)M.nnz()) return D;
  std::sort(offs.begin(), offs.end());
  const int nd = (int)offs.size();
  std::vector<double> full((size_t)nd * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = M.ptr[i]; e < M.ptr[i + 1]; ++e) {
      const int64_t o = (int64_t)M.idx[e] - i;
      const int d = (int)(std::find(offs.begin(), offs.end(), o) - offs.begin());
      full[(size_t)d * n + i] += M.val[e];
    }
  // exact symmetry: a_{i,i+o} == a_{i+o,i} for every upper diagonal o
  bool sym = true;
  for (int d = 0; d < nd && sym; ++d) {
    if (offs[d] <= 0) continue;
    const auto it = std::find(offs.begin(), offs.end(), -offs[d]);
    if (it == offs.end()) {
      sym = false;
      break;
    }
    const int dl = (int)(it - offs.begin());
    for (int64_t i = 0; i + offs[d] < n; ++i)
      if (full[(size_t)d * n + i] != full[(size_t)dl * n + i + offs[d]]) {
        sym = false;
        break;
      }
  }
  D.ndiag = nd;
  std::vector<int> stored_of(nd, -1);
  for (int d = 0; d < nd; ++d) {
    D.off[d] = (int32_t)offs[d];
    if (sym && offs[d] > 0) continue;
    stored_of[d] = D.nstored++;
  }
  for (int d = 0; d < nd; ++d) {
    if (stored_of[d] >= 0) {
      D.src[d] = stored_of[d];
      D.shift[d] = 0;
    } else {
      const int dl = (int)(std::find(offs.begin(), offs.end(), -offs[d]) - offs.begin());
      D.src[d] = stored_of[dl];
      D.shift[d] = (int32_t)offs[d];
    }
  }
  D.val.resize((size_t)D.nstored * n);
  for (int d = 0; d < nd; ++d)
    if (stored_of[d] >= 0)
      std::copy(full.begin() + (size_t)d * n, full.begin() + (size_t)(d + 1) * n,
                D.val.begin() + (size_t)stored_of[d] * n);
  return D;
}

}  // namespace amgsym

using namespace amgsym;

#define API_BEGIN try {
#define API_END                                          \
  }                                                      \
  catch (const amgsym::Error& e) {                       \
    amgsym::set_last_error(e.msg);                       \
    return e.code;                                       \
  }                                                      \
  catch (const std::bad_alloc&) {                        \
    amgsym::set_last_error("host allocation failed");    \
    return AMGSYM_ERR_OOM;                               \
  }                                                      \
  return AMGSYM_OK;

extern "C" amgsym_status amgsym_setup(amgsym_t h, const amgsym_opts* opts) {
  API_BEGIN
  if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
  amgsym_opts o;
  amgsym_opts_default(&o);
  if (opts) o = *opts;
  if (o.nu < 1 || o.nu > 8) fail(AMGSYM_ERR_ARG, "nu must be in [1, 8]");
  if (o.fuse_rows < 0 || o.dia_max_diag < 0 || o.halo_kb < 0)
    fail(AMGSYM_ERR_ARG, "fuse_rows, dia_max_diag and halo_kb must be >= 0");
  if (o.fsai_max_lower < 1 || o.fsai_max_lower > 32 || o.fsai_max_lower_coarse < 1 || o.fsai_max_lower_coarse > 32)
    fail(AMGSYM_ERR_ARG, "fsai_max_lower and fsai_max_lower_coarse must be in [1, 32]");
  if (o.coarse_max < 1 || o.coarse_max > kDenseLimit) fail(AMGSYM_ERR_ARG, "coarse_max out of range");
  if (o.max_levels < 1) fail(AMGSYM_ERR_ARG, "max_levels must be >= 1");
  if ((o.precisions & 7) == 0) fail(AMGSYM_ERR_ARG, "precisions mask is empty");
  if (o.zmarch != 0 && o.zmarch != 1) fail(AMGSYM_ERR_ARG, "zmarch must be 0 or 1");
  if (o.sell != 0 && o.sell != 1) fail(AMGSYM_ERR_ARG, "sell must be 0 or 1");
  if (o.amgr_sym_ac != 0 && o.amgr_sym_ac != 1) fail(AMGSYM_ERR_ARG, "amgr_sym_ac must be 0 or 1");
  if (o.lambda_device != 0 && o.lambda_device != 1) fail(AMGSYM_ERR_ARG, "lambda_device must be 0 or 1");
  if (o.amgr && (o.amgr_distance < 1 || o.amgr_distance > 4 || o.amgr_interp_max < 1))
    fail(AMGSYM_ERR_ARG, "amgr_distance must be in [1, 4] and amgr_interp_max >= 1");
  device_free(h);
  h->have_hierarchy = false;
  h->opts = o;
  build_hierarchy(h->Ainn, o, h->H);
  for (HostLevel& L : h->H.levels) {
    L.Adia = build_dia(L.A, o.dia_max_diag);
    L.Gdia = build_dia(L.G, o.dia_max_diag);
    L.Gtdia = build_dia(L.Gt, o.dia_max_diag);
  }
  h->amgr.reset();
  if (o.amgr) build_amgr(h, o);
  h->have_hierarchy = true;
  if (!o.host_only) device_upload(h);
  API_END
}

extern "C" int32_t amgsym_num_levels(amgsym_t h) {
  if (!h || !h->have_hierarchy) return 0;
  return (int32_t)h->H.levels.size();
}

extern "C" amgsym_status amgsym_level_sizes(amgsym_t h, int32_t level, int64_t* rows, int64_t* nnz_A,
                                            int64_t* nnz_P, int64_t* cols_P, int64_t* nnz_G,
                                            double* omega) {
  API_BEGIN
  if (!h || !h->have_hierarchy) fail(AMGSYM_ERR_STATE, "no hierarchy (call amgsym_setup)");
  if (level < 0 || level >= (int32_t)h->H.levels.size()) fail(AMGSYM_ERR_ARG, "level out of range");
  const HostLevel& L = h->H.levels[level];
  if (rows) *rows = L.A.rows;
  if (nnz_A) *nnz_A = L.A.nnz();
  if (nnz_P) *nnz_P = L.P.nnz();
  if (cols_P) *cols_P = L.P.cols;
  if (nnz_G) *nnz_G = L.G.nnz();
  if (omega) *omega = L.omega;
  API_END
}

extern "C" amgsym_status amgsym_get_level_matrix(amgsym_t h, int32_t level, int32_t which,
                                                 int64_t* rowptr, int32_t* colidx, double* vals) {
  API_BEGIN
  if (!h || !h->have_hierarchy) fail(AMGSYM_ERR_STATE, "no hierarchy (call amgsym_setup)");
  if (level < 0 || level >= (int32_t)h->H.levels.size()) fail(AMGSYM_ERR_ARG, "level out of range");
  const HostLevel& L = h->H.levels[level];
  const Csr* M = which == 0 ? &L.A : which == 1 ? &L.P : which == 2 ? &L.G : nullptr;
  if (!M) fail(AMGSYM_ERR_ARG, "which must be 0 (A), 1 (P) or 2 (G)");
  if (M->rows == 0) fail(AMGSYM_ERR_ARG, "matrix absent on this level");
  if (!rowptr || !colidx || !vals) fail(AMGSYM_ERR_ARG, "NULL output");
  std::memcpy(rowptr, M->ptr.data(), sizeof(int64_t) * M->ptr.size());
  std::memcpy(colidx, M->idx.data(), sizeof(int32_t) * M->idx.size());
  std::memcpy(vals, M->val.data(), sizeof(double) * M->val.size());
  API_END
}

extern "C" amgsym_status amgsym_level_dia(amgsym_t h, int32_t level, int32_t which, int32_t* ndiag,
                                         int32_t* nstored, int32_t* offsets) {
  API_BEGIN
  if (!h || !h->have_hierarchy) fail(AMGSYM_ERR_STATE, "no hierarchy (call amgsym_setup)");
  if (level < 0 || level >= (int32_t)h->H.levels.size()) fail(AMGSYM_ERR_ARG, "level out of range");
  const HostLevel& L = h->H.levels[level];
  const Dia* D = which == 0 ? &L.Adia : which == 2 ? &L.Gdia : which == 3 ? &L.Gtdia : nullptr;
  if (!D) fail(AMGSYM_ERR_ARG, "which must be 0 (A), 2 (G) or 3 (G^T)");
  if (ndiag) *ndiag = D->ndiag;
  if (nstored) *nstored = D->nstored;
  if (offsets)
    for (int d = 0; d < AMGSYM_MAX_DIAG; ++d) offsets[d] = d < D->ndiag ? D->off[d] : 0;
  API_END
}
