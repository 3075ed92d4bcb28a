// Host setup of AMGR, the paper's multigrid reduction (Sec. 3.2).
//
// AMGR works on the full operator A.  Its first level reduces A to the
// "populated interface": the interface unknowns (those coupled to another
// mirror copy) plus inner unknowns chosen by an aggressive coarsening
// (Alg. "popul"): classical strength of A_inn, the graph T of its strong
// connections between inner points, and a maximal independent set of T^k
// (no two selected points within distance k; every inner point within
// distance k of one).  The same points are coarse in every copy, so the
// inner block K-bar = I (x) K and the prolongation P = I (x) P_b with
// P_b = [W; I] (eq. "amgreduction") are the same for every copy: in the
// transformed basis of Alg. 1 they act on all 2^s blocks at once (SpMM).
// W is extended+i interpolation.  The paper's best configuration is k = 2
// with DPLS + energy minimisation; with extended+i, k = 1 converges as the
// paper's AMGR does (9-11 PCG iterations on the 32^3 model problem, s >= 1)
// and k = 2 does not (22-26), so k = 1 is the default.
//
// The top-level smoother is the block FSAI of eq. "topsmoother": the FSAI of
// K on the fine points (shared by every copy) and an FSAI of C-bar on the
// coarse points, here with a diagonal pattern (damped Jacobi).  The reduced
// operator A_c = P^T A P (eq. "structAc") keeps the dyadic structure of eq.
// "struct_2sym" (its blocks are P_b^T H_m P_b); it is assembled as one matrix
// over the full coarse domain (copy index fastest) and gets a standard AMG.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <random>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace amgsym {

// Maximal independent set of the inner points at distance `dist` in the
// symmetric graph T (strong connections in either direction between inner
// points): points are taken in a seeded random order; a point not yet
// excluded is selected and excludes every point within distance dist.
static std::vector<uint8_t> mis_distance(const Csr& A, const std::vector<uint8_t>& strong,
                                         const std::vector<uint8_t>& inner, int dist, uint64_t seed) {
  const int64_t n = A.rows;
  // T = strong pattern symmetrised, inner points only
  std::vector<uint8_t> keep(A.nnz(), 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) keep[e] = strong[e] && inner[i] && inner[A.idx[e]];
  const Csr S = pattern_of(A, keep);
  const Csr ST = transpose(S);
  std::vector<int64_t> order;
  for (int64_t i = 0; i < n; ++i)
    if (inner[i]) order.push_back(i);
  std::mt19937_64 rng(seed);
  std::shuffle(order.begin(), order.end(), rng);
  std::vector<uint8_t> state(n, 0);  // 0 undecided, 1 selected, 2 excluded
  std::vector<int64_t> frontier, next, touched;
  std::vector<int32_t> seen(n, -1);
  int32_t stamp = 0;
  for (int64_t i : order) {
    if (state[i] != 0) continue;
    state[i] = 1;
    ++stamp;
    frontier.assign(1, i);
    seen[i] = stamp;
    for (int d = 0; d < dist; ++d) {
      next.clear();
      for (int64_t u : frontier) {
        for (const Csr* G : {(const Csr*)&S, &ST})
          for (int64_t e = G->ptr[u]; e < G->ptr[u + 1]; ++e) {
            const int32_t v = G->idx[e];
            if (seen[v] == stamp) continue;
            seen[v] = stamp;
            if (state[v] == 0) state[v] = 2;
            next.push_back(v);
          }
      }
      frontier.swap(next);
    }
  }
  std::vector<uint8_t> sel(n, 0);
  for (int64_t i = 0; i < n; ++i) sel[i] = state[i] == 1;
  return sel;
}

static double lambda_max_diag_scaled(const Csr& A, const std::vector<int64_t>& rows, uint64_t seed) {
  // power iteration on D^{-1/2} A D^{-1/2} restricted to `rows` (a subset)
  const int64_t m = (int64_t)rows.size();
  if (m == 0) return 1.0;
  std::vector<int64_t> pos(A.rows, -1);
  for (int64_t k = 0; k < m; ++k) pos[rows[k]] = k;
  std::vector<double> dinv(m), v(m), w(m);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < m; ++k) {
    double d = 0.0;
    for (int64_t e = A.ptr[rows[k]]; e < A.ptr[rows[k] + 1]; ++e)
      if (A.idx[e] == rows[k]) d = A.val[e];
    dinv[k] = d > 0.0 ? 1.0 / std::sqrt(d) : 0.0;
  }
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (auto& x : v) x = U(rng);
  double lam = 1.0;
  for (int it = 0; it < 30; ++it) {
    double nv = 0.0;
    for (double x : v) nv += x * x;
    nv = std::sqrt(nv);
    if (nv == 0.0) break;
    for (auto& x : v) x /= nv;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
      double s = 0.0;
      const int64_t r = rows[k];
      for (int64_t e = A.ptr[r]; e < A.ptr[r + 1]; ++e) {
        const int64_t q = pos[A.idx[e]];
        if (q >= 0) s += A.val[e] * dinv[q] * v[q];
      }
      w[k] = dinv[k] * s;
    }
    double num = 0.0;
    for (int64_t k = 0; k < m; ++k) num += v[k] * w[k];
    lam = num;
    v.swap(w);
  }
  return lam;
}

void build_amgr(amgsym_problem* p, const amgsym_opts& o) {
  auto H = std::make_shared<HostAmgr>();
  const Csr& A = p->Ainn;  // rows sorted
  const int64_t n_b = A.rows;
  const int32_t nb = p->nb;
  // interface points: base rows with a coupling to another copy
  std::vector<uint8_t> inner(n_b, 1);
  for (int32_t r : p->irow) inner[r] = 0;
  const std::vector<uint8_t> strong = strength(A, o.strength_theta);
  const std::vector<uint8_t> sel = mis_distance(A, strong, inner, o.amgr_distance, o.seed + 101);
  H->cf.assign(n_b, -1);
  for (int64_t i = 0; i < n_b; ++i)
    if (!inner[i] || sel[i]) H->cf[i] = 1;
  // P_b = [W; I]: extended+i with the populated splitting
  H->Pb = ext_i_interp(A, strong, H->cf, o.interp_trunc, o.amgr_interp_max);
  H->Rb = transpose(H->Pb);
  H->n_cb = (int32_t)H->Pb.cols;
  // K = A_inn[F, F] and its FSAI, embedded in the base numbering
  std::vector<int32_t> fidx(n_b, -1);
  std::vector<int64_t> frows, crows;
  for (int64_t i = 0; i < n_b; ++i) {
    if (H->cf[i] < 0) {
      fidx[i] = (int32_t)frows.size();
      frows.push_back(i);
    } else {
      crows.push_back(i);
    }
  }
  Csr K;
  K.rows = K.cols = (int64_t)frows.size();
  K.ptr.assign(K.rows + 1, 0);
  for (int64_t k = 0; k < K.rows; ++k) {
    const int64_t i = frows[k];
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
      if (fidx[A.idx[e]] >= 0) {
        K.idx.push_back(fidx[A.idx[e]]);
        K.val.push_back(A.val[e]);
      }
    K.ptr[k + 1] = (int64_t)K.idx.size();
  }
  const Csr GKf = fsai(K, o.fsai_max_lower);
  const Csr GKft = transpose(GKf);
  const double lamK = K.rows > 0 ? lambda_max_GAGt(K, GKf, GKft, o.seed + 202) : 1.0;
  H->omegaK = lamK > 0.0 ? o.omega_scale / lamK : 1.0;
  H->GK.rows = H->GK.cols = n_b;
  H->GK.ptr.assign(n_b + 1, 0);
  for (int64_t i = 0; i < n_b; ++i) {
    if (fidx[i] >= 0) {
      const int64_t k = fidx[i];
      for (int64_t e = GKf.ptr[k]; e < GKf.ptr[k + 1]; ++e) {
        H->GK.idx.push_back((int32_t)frows[GKf.idx[e]]);
        H->GK.val.push_back(GKf.val[e]);
      }
    }
    H->GK.ptr[i + 1] = (int64_t)H->GK.idx.size();
  }
  H->GKt = transpose(H->GK);
  // coarse-point smoother: the FSAI of C-bar with a diagonal pattern, i.e.
  // omega_C / a_ll, omega_C from lambda_max of D^{-1/2} C D^{-1/2}
  const double lamC = lambda_max_diag_scaled(A, crows, o.seed + 303);
  const double omegaC = lamC > 0.0 ? o.omega_scale / lamC : 1.0;
  H->jdC.assign(n_b, 0.0);
  for (int64_t i : crows) {
    double d = 0.0;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
      if (A.idx[e] == i) d = A.val[e];
    H->jdC[i] = d > 0.0 ? omegaC / d : 0.0;
  }
  // A_c = P^T A P, block (p, q) = P_b^T H_{p XOR q} P_b.  H_0 = A_inn; the
  // blocks H_m (m >= 1) come back from the stored interface couplings
  // A_out,i = sum_m sign(i, m) H_m by the inverse Walsh-Hadamard transform;
  // they live on interface rows and columns, which are coarse points with
  // unit rows in P_b, so P_b^T H_m P_b = H_m on their coarse indices.
  const Csr AP = spgemm(A, H->Pb);
  Csr Ac0 = spgemm(H->Rb, AP);
  sort_rows(Ac0);
  std::vector<int32_t> cmap(n_b, -1);
  {
    int32_t c = 0;
    for (int64_t i = 0; i < n_b; ++i)
      if (H->cf[i] > 0) cmap[i] = c++;
  }
  const int64_t ne = (int64_t)p->irow.size();
  // the transformed-basis form: the fine couplings at coarse indices (cmap
  // is increasing, so the entries stay sorted by (row, column))
  H->cirow.resize(ne);
  H->cicol.resize(ne);
  for (int64_t e = 0; e < ne; ++e) {
    H->cirow[e] = cmap[p->irow[e]];
    H->cicol[e] = cmap[p->icol[e]];
    if (H->cirow[e] < 0 || H->cicol[e] < 0) fail(AMGSYM_ERR_STATE, "AMGR: an interface point is not coarse");
  }
  H->civals = p->ivals;
  // per coarse row: (coarse col, m, value) of the couplings to other copies
  std::vector<std::vector<std::tuple<int32_t, int32_t, double>>> cross(H->n_cb);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t rc = cmap[p->irow[e]], cc = cmap[p->icol[e]];
    for (int32_t m = 1; m < nb; ++m) {
      double hm = 0.0;
      for (int32_t i = 0; i < nb; ++i)
        hm += ((__builtin_popcount((unsigned)(i & m)) & 1) ? -1.0 : 1.0) * p->ivals[(size_t)e * nb + i];
      hm /= (double)nb;
      if (hm != 0.0) cross[rc].push_back({cc, m, hm});
    }
  }
  // row (lc, j) of A_c: row lc of Ac0 in copy j, then the couplings to the
  // copies j XOR m (no column repeats: those land in other copies)
  const int64_t nc = (int64_t)H->n_cb * nb;
  Csr Ac;
  Ac.rows = Ac.cols = nc;
  Ac.ptr.assign(nc + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nc; ++r) {
    const int64_t lc = r / nb;
    Ac.ptr[r + 1] = (Ac0.ptr[lc + 1] - Ac0.ptr[lc]) + (int64_t)cross[lc].size();
  }
  for (int64_t r = 0; r < nc; ++r) Ac.ptr[r + 1] += Ac.ptr[r];
  Ac.idx.resize(Ac.ptr[nc]);
  Ac.val.resize(Ac.ptr[nc]);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nc; ++r) {
    const int64_t lc = r / nb;
    const int32_t j = (int32_t)(r % nb);
    int64_t w = Ac.ptr[r];
    for (int64_t e = Ac0.ptr[lc]; e < Ac0.ptr[lc + 1]; ++e) {
      Ac.idx[w] = Ac0.idx[e] * nb + j;
      Ac.val[w++] = Ac0.val[e];
    }
    for (const auto& t : cross[lc]) {
      Ac.idx[w] = std::get<0>(t) * nb + (j ^ std::get<1>(t));
      Ac.val[w++] = std::get<2>(t);
    }
  }
  sort_rows(Ac);
  H->Ac0 = std::move(Ac0);
  // the coarse problem: s = 0, its own standard AMG hierarchy, whose finest
  // level takes over A_c (its Ainn keeps only the shape)
  auto* cp = new amgsym_problem();
  cp->n = nc;
  cp->n_b = nc;
  cp->s = 0;
  cp->nb = 1;
  cp->Ainn.rows = cp->Ainn.cols = nc;
  cp->perm.resize(nc);
  std::iota(cp->perm.begin(), cp->perm.end(), 0);
  cp->singular = p->singular;
  cp->opts = o;
  cp->opts.amgr = 0;
  cp->opts.dia_max_diag = 0;
  build_hierarchy(std::move(Ac), cp->opts, cp->H);
  cp->have_hierarchy = true;
  H->coarse = std::shared_ptr<amgsym_problem>(cp, [](amgsym_problem* q) { amgsym_destroy(q); });
  p->amgr = H;
}

}  // namespace amgsym
