// LRCAMG(k): the low-rank corrected AMG of Sec. 2.2 (Thm. "correction_nonfact",
// eqs. "Ydef_AMG", "LRC_AMG", "LRCAMG") and the GMRES solve it is used with
// (the paper's Table "lrcamg").
//
// For every block i the preconditioner I (x) M_inn^{-1} (one AMG hierarchy of
// A_inn for all blocks) ignores the interface coupling A_out,i.  With
// X = M_inn^{-1} A^_i and Y = I - X = U Sigma V^T (right and left
// eigenvectors, V^T U = I), the theorem gives A^_i^{-1} = (I + U Theta V^T)
// M_inn^{-1} with Theta = (Sigma^{-1} - I)^{-1}; keeping the k eigenpairs of
// the smallest eigenvalues lambda of X (the ones that slow a Krylov method
// down) gives the rank-k correction of eq. "LRC_AMG", which maps those
// eigenvalues of the preconditioned operator to 1.  With Sigma = I - Lambda,
// Theta_t = (1 - lambda_t) / lambda_t.
//
// Computing the pairs.  X is self-adjoint in the A^_i inner product, so
// Lanczos in that inner product (full reorthogonalisation, both Gram-Schmidt
// passes) gives A^_i-orthonormal Ritz vectors u; then v = A^_i u is the left
// eigenvector that pairs with u (v^T X = lambda v^T, v^T u = 1).  Every block
// runs its own Lanczos as one column of the interleaved multi-column layout,
// so each step is one reduced SpMM and one V-cycle for all blocks at once.
//
// Application, per column of block i: z = w + U_i (Theta_i V_i^T w) with
// w = M_inn^{-1} r: k dots and k updates (k_krylov.cu).  The correction is not
// symmetric, hence GMRES (restarted, right-preconditioned, classical
// Gram-Schmidt with one reorthogonalisation) as in the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "device.h"
#include "internal.h"
#include "solver.h"

namespace amgsym {

namespace {

// Device scratch freed on scope exit.
struct DevBuf {
  double* p = nullptr;
  DevBuf() = default;
  explicit DevBuf(int64_t count) {
    if (count > 0) CK(cudaMalloc(&p, sizeof(double) * (size_t)count));
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

void to_host(double* dst, const double* src, int64_t count, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

void to_dev(double* dst, const double* src, int64_t count, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)count, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
}

// Eigen-decomposition of a small symmetric matrix (m x m, row-major) by
// cyclic Jacobi rotations: on return the diagonal of T holds the eigenvalues
// and column t of Q the eigenvector of T[t][t].
void jacobi_eig(std::vector<double>& T, std::vector<double>& Q, int m) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double v = T[(size_t)i * m + j] * T[(size_t)i * m + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = T[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double app = T[(size_t)p * m + p], aqq = T[(size_t)q * m + q];
        // the rotation angle that zeroes (p, q): tan(2 phi) = 2 apq / (aqq - app)
        const double theta = 0.5 * (aqq - app) / apq;
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < m; ++r) {  // T <- T J (columns p, q)
          const double trp = T[(size_t)r * m + p], trq = T[(size_t)r * m + q];
          T[(size_t)r * m + p] = c * trp - s * trq;
          T[(size_t)r * m + q] = s * trp + c * trq;
        }
        for (int r = 0; r < m; ++r) {  // T <- J^T T (rows p, q)
          const double tpr = T[(size_t)p * m + r], tqr = T[(size_t)q * m + r];
          T[(size_t)p * m + r] = c * tpr - s * tqr;
          T[(size_t)q * m + r] = s * tpr + c * tqr;
        }
        for (int r = 0; r < m; ++r) {  // Q <- Q J
          const double qrp = Q[(size_t)r * m + p], qrq = Q[(size_t)r * m + q];
          Q[(size_t)r * m + p] = c * qrp - s * qrq;
          Q[(size_t)r * m + q] = s * qrp + c * qrq;
        }
      }
  }
}

// z = w + U (Theta V^T w) per column (block c % nb), in place on z.
void apply_lrc(Device* D, int32_t C, double* z, double* part, double* Hd, cudaStream_t st) {
  if (D->lrc_k <= 0) return;
  const int64_t vs = D->n_b * D->nb;
  launch_mdot(D->lrc_V, vs, D->nb, D->lrc_k, z, D->n_b, C, part, Hd, st);
  launch_maxpy(D->lrc_U, vs, D->nb, D->lrc_k, Hd, 1.0, z, D->n_b, C, st);
  check_launch();
}

}  // namespace

// Lanczos in the A^_i inner product on X = M_inn^{-1} A^_i for all blocks at
// once; keeps the k Ritz pairs of the smallest Ritz values.
static void lrc_setup(amgsym_t h, int32_t k, int32_t steps, uint64_t seed, cudaStream_t st) {
  Device* D = require_dev(h);
  D->lrc_k = 0;
  D->lrc_U = D->lrc_V = nullptr;  // the old arrays stay owned until device_free
  D->lrc_theta.clear();
  if (k == 0) return;
  const int32_t nb = D->nb, C = nb;
  const int64_t n_b = D->n_b, len = n_b * C;
  const int m = steps;
  ensure_work(D, 1, VEC_F64);
  Ctx c{D, C, VEC_F64, VAL_F64, false, st};
  c.fuse = true;
  DevBuf Q((int64_t)(m + 1) * len), AQ((int64_t)(m + 1) * len), w(len), part((int64_t)mdot_blocks(n_b, C) * (m + 1) * C),
      Hd((int64_t)(m + 1) * C), sd(C);
  // start vector: uniform[-1, 1] from the seed
  {
    std::vector<double> q0((size_t)len);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (auto& v : q0) v = U(rng);
    to_dev(Q.p, q0.data(), len, st);
  }
  std::vector<double> hh((size_t)(m + 1) * C), sv(C);
  auto normalise = [&](double* q, double* aq) {  // q, aq *= 1 / sqrt(q^T A^ q), per column
    launch_mdot(q, 0, C, 1, aq, n_b, C, part.p, Hd.p, st);
    check_launch();
    to_host(hh.data(), Hd.p, C, st);
    for (int j = 0; j < C; ++j) sv[j] = hh[j] > 0.0 ? 1.0 / std::sqrt(hh[j]) : 0.0;
    to_dev(sd.p, sv.data(), C, st);
    launch_colscale(q, sd.p, q, n_b, C, st);
    launch_colscale(aq, sd.p, aq, n_b, C, st);
    check_launch();
    return hh;
  };
  spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, Q.p, AQ.p, 1.0, 0.0, nullptr, true, nullptr);
  normalise(Q.p, AQ.p);
  std::vector<double> alpha((size_t)m * C, 0.0), beta((size_t)m * C, 0.0);
  std::vector<int> mc(C, m);  // Lanczos steps taken per column (an invariant subspace ends it early)
  for (int j = 0; j < m; ++j) {
    double* aqj = AQ.p + (int64_t)j * len;
    vcycle_apply(c, aqj, w.p);  // w = M_inn^{-1} A^ q_j
    check_launch();
    std::vector<double> h_sum((size_t)(j + 1) * C, 0.0);
    for (int pass = 0; pass < 2; ++pass) {  // w -= Q (AQ^T w), twice
      launch_mdot(AQ.p, len, C, j + 1, w.p, n_b, C, part.p, Hd.p, st);
      launch_maxpy(Q.p, len, C, j + 1, Hd.p, -1.0, w.p, n_b, C, st);
      check_launch();
      to_host(hh.data(), Hd.p, (int64_t)(j + 1) * C, st);
      for (int64_t t = 0; t < (int64_t)(j + 1) * C; ++t) h_sum[t] += hh[t];
    }
    for (int col = 0; col < C; ++col) alpha[(size_t)j * C + col] = h_sum[(size_t)j * C + col];
    double* qn = Q.p + (int64_t)(j + 1) * len;
    double* aqn = AQ.p + (int64_t)(j + 1) * len;
    CK(cudaMemcpyAsync(qn, w.p, sizeof(double) * (size_t)len, cudaMemcpyDeviceToDevice, st));
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, qn, aqn, 1.0, 0.0, nullptr, true, nullptr);
    const std::vector<double> b2 = normalise(qn, aqn);
    for (int col = 0; col < C; ++col) {
      double amax = 0.0;
      for (int i = 0; i <= j; ++i) amax = std::max(amax, std::fabs(alpha[(size_t)i * C + col]));
      const double b = b2[col] > 0.0 ? std::sqrt(b2[col]) : 0.0;
      beta[(size_t)j * C + col] = b;
      if (mc[col] == m && !(b > 1e-10 * amax)) mc[col] = j + 1;  // invariant subspace: T is complete
    }
  }
  // Ritz pairs per column; the k smallest (or all the column has)
  std::vector<double> theta((size_t)C * k, 0.0), Y((size_t)m * k * C, 0.0), Yv((size_t)m * k * C, 0.0);
  for (int col = 0; col < C; ++col) {
    const int mm = mc[col];
    std::vector<double> T((size_t)mm * mm, 0.0), V;
    for (int i = 0; i < mm; ++i) {
      T[(size_t)i * mm + i] = alpha[(size_t)i * C + col];
      if (i + 1 < mm) T[(size_t)i * mm + i + 1] = T[(size_t)(i + 1) * mm + i] = beta[(size_t)i * C + col];
    }
    jacobi_eig(T, V, mm);
    std::vector<int> order(mm);
    for (int i = 0; i < mm; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return T[(size_t)a * mm + a] < T[(size_t)b * mm + b]; });
    for (int t = 0; t < k && t < mm; ++t) {
      const int e = order[t];
      const double th = T[(size_t)e * mm + e];
      theta[(size_t)col * k + t] = th;
      const double Th = th > 0.0 ? (1.0 - th) / th : 0.0;  // Theta_t of eq. "LRC_AMG"
      for (int i = 0; i < mm; ++i) {
        Y[((size_t)t * m + i) * C + col] = V[(size_t)i * mm + e];
        Yv[((size_t)t * m + i) * C + col] = Th * V[(size_t)i * mm + e];
      }
    }
  }
  // U_t = Q Y_t and V_t = Theta_t A^ U_t = (A^ Q) Theta_t Y_t, stored [k][n_b][nb]
  double* U = nullptr;
  double* Vv = nullptr;
  CK(cudaMalloc(&U, sizeof(double) * (size_t)k * len));
  D->owned.push_back(U);
  CK(cudaMalloc(&Vv, sizeof(double) * (size_t)k * len));
  D->owned.push_back(Vv);
  CK(cudaMemsetAsync(U, 0, sizeof(double) * (size_t)k * len, st));
  CK(cudaMemsetAsync(Vv, 0, sizeof(double) * (size_t)k * len, st));
  for (int t = 0; t < k; ++t) {
    to_dev(Hd.p, Y.data() + (size_t)t * m * C, (int64_t)m * C, st);
    launch_maxpy(Q.p, len, C, m, Hd.p, 1.0, U + (int64_t)t * len, n_b, C, st);
    to_dev(Hd.p, Yv.data() + (size_t)t * m * C, (int64_t)m * C, st);
    launch_maxpy(AQ.p, len, C, m, Hd.p, 1.0, Vv + (int64_t)t * len, n_b, C, st);
    check_launch();
  }
  CK(cudaStreamSynchronize(st));
  D->lrc_k = k;
  D->lrc_U = U;
  D->lrc_V = Vv;
  D->lrc_theta = theta;
}

// Restarted right-preconditioned GMRES on the reduced system, every column
// its own Arnoldi process (one launch per step for all columns).
static amgsym_status gmres_impl(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                const amgsym_solve_opts* sopts, int32_t restart, int32_t use_lrc, cudaStream_t st,
                                amgsym_solve_info* info) {
  Device* D = require_dev(h);
  amgsym_solve_opts o;
  amgsym_solve_opts_default(&o);
  if (sopts) o = *sopts;
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  if (ld < h->n || !b_dev || !x_dev) fail(AMGSYM_ERR_ARG, "bad vectors or ld");
  if (o.precision != AMGSYM_PREC_FP64) fail(AMGSYM_ERR_ARG, "the GMRES solve runs in FP64 (AMGSYM_PREC_FP64)");
  if (!(o.tol > 0.0) || o.maxit < 1) fail(AMGSYM_ERR_ARG, "bad tolerance or maxit");
  if (restart < 1 || restart > 500) fail(AMGSYM_ERR_ARG, "restart must be in [1, 500]");
  if (use_lrc && D->lrc_k <= 0) fail(AMGSYM_ERR_STATE, "no low-rank correction: call amgsym_lrc_setup first");
  ensure_work(D, nrhs, VEC_F64);
  const int32_t nb = D->nb, C = nrhs * nb;
  const int64_t n_b = D->n_b, len = n_b * C;
  const int m = restart;
  Ctx c{D, C, VEC_F64, VAL_F64, o.finest_hat != 0, st};
  c.fuse = true;
  DevBuf V((int64_t)(m + 1) * len), Z((int64_t)m * len), w(len),
      part((int64_t)mdot_blocks(n_b, C) * std::max(m + 1, D->lrc_k + 1) * C), Hd((int64_t)(m + 1) * C), sd(C);
  double* bh = D->bh;
  double* xh = D->xh;
  launch_transform_fwd(b_dev, nrhs, ld, D->perm, n_b, D->s, bh, VEC_F64, st);
  check_launch();
  if (D->singular) launch_sub_block0_mean(bh, n_b, nrhs, nb, D->sc_out.partials, D->sc_out.partial_cap, st);
  if (o.use_x0)
    launch_transform_fwd(x_dev, nrhs, ld, D->perm, n_b, D->s, xh, VEC_F64, st);
  else
    CK(cudaMemsetAsync(xh, 0, sizeof(double) * (size_t)len, st));
  check_launch();
  std::vector<double> hv((size_t)(m + 1) * C), bn2(nrhs, 0.0), sv(C);
  launch_mdot(bh, 0, C, 1, bh, n_b, C, part.p, Hd.p, st);
  check_launch();
  to_host(hv.data(), Hd.p, C, st);
  for (int col = 0; col < C; ++col) bn2[col / nb] += hv[col];
  auto relres_of = [&](const std::vector<double>& col2, std::vector<double>& rel) {
    rel.assign(nrhs, 0.0);
    for (int col = 0; col < C; ++col) rel[col / nb] += col2[col];
    bool ok = true;
    for (int r = 0; r < nrhs; ++r) {
      rel[r] = bn2[r] > 0.0 ? std::sqrt(rel[r] / bn2[r]) : 0.0;
      if (!(rel[r] <= o.tol)) ok = false;
    }
    return ok;
  };
  std::vector<double> rel;
  int total = 0;
  bool converged = false;
  // Hessenberg (after rotations), rotations and right-hand side per column
  std::vector<double> Hc((size_t)(m + 1) * m * C), cs((size_t)m * C), sn((size_t)m * C), g((size_t)(m + 1) * C);
  while (true) {
    // r = b^ - A^ x^ -> V_0 = r / ||r|| per column
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, xh, V.p, -1.0, 1.0, bh, true, nullptr);
    launch_mdot(V.p, 0, C, 1, V.p, n_b, C, part.p, Hd.p, st);
    check_launch();
    std::vector<double> r2(C);
    to_host(r2.data(), Hd.p, C, st);
    converged = relres_of(r2, rel);
    if (converged || total >= o.maxit) break;
    std::fill(g.begin(), g.end(), 0.0);
    for (int col = 0; col < C; ++col) {
      const double beta = std::sqrt(std::max(0.0, r2[col]));
      g[col] = beta;
      sv[col] = beta > 0.0 ? 1.0 / beta : 0.0;
    }
    to_dev(sd.p, sv.data(), C, st);
    launch_colscale(V.p, sd.p, V.p, n_b, C, st);
    int j = 0;
    for (; j < m && total < o.maxit; ++j, ++total) {
      double* vj = V.p + (int64_t)j * len;
      double* zj = Z.p + (int64_t)j * len;
      vcycle_apply(c, vj, zj);  // z_j = P v_j (eq. "LRCAMG")
      if (use_lrc) apply_lrc(D, C, zj, part.p, Hd.p, st);
      spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, zj, w.p, 1.0, 0.0, nullptr, true, nullptr);
      std::vector<double> hsum((size_t)(j + 1) * C, 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        launch_mdot(V.p, len, C, j + 1, w.p, n_b, C, part.p, Hd.p, st);
        launch_maxpy(V.p, len, C, j + 1, Hd.p, -1.0, w.p, n_b, C, st);
        check_launch();
        to_host(hv.data(), Hd.p, (int64_t)(j + 1) * C, st);
        for (int64_t t = 0; t < (int64_t)(j + 1) * C; ++t) hsum[t] += hv[t];
      }
      launch_mdot(w.p, 0, C, 1, w.p, n_b, C, part.p, Hd.p, st);
      check_launch();
      std::vector<double> hn2(C);
      to_host(hn2.data(), Hd.p, C, st);
      std::vector<double> res2(C);
      for (int col = 0; col < C; ++col) {
        std::vector<double> hc(j + 2);
        for (int i = 0; i <= j; ++i) hc[i] = hsum[(size_t)i * C + col];
        hc[j + 1] = std::sqrt(std::max(0.0, hn2[col]));
        sv[col] = hc[j + 1] > 0.0 ? 1.0 / hc[j + 1] : 0.0;
        for (int i = 0; i < j; ++i) {  // earlier rotations
          const double a = hc[i], b = hc[i + 1];
          hc[i] = cs[(size_t)i * C + col] * a + sn[(size_t)i * C + col] * b;
          hc[i + 1] = -sn[(size_t)i * C + col] * a + cs[(size_t)i * C + col] * b;
        }
        const double rr = std::hypot(hc[j], hc[j + 1]);
        const double cj = rr > 0.0 ? hc[j] / rr : 1.0, sj = rr > 0.0 ? hc[j + 1] / rr : 0.0;
        cs[(size_t)j * C + col] = cj;
        sn[(size_t)j * C + col] = sj;
        hc[j] = rr;
        const double gj = g[(size_t)j * C + col];
        g[(size_t)j * C + col] = cj * gj;
        g[(size_t)(j + 1) * C + col] = -sj * gj;
        for (int i = 0; i <= j; ++i) Hc[((size_t)i * m + j) * C + col] = hc[i];
        res2[col] = g[(size_t)(j + 1) * C + col] * g[(size_t)(j + 1) * C + col];
      }
      to_dev(sd.p, sv.data(), C, st);
      launch_colscale(w.p, sd.p, V.p + (int64_t)(j + 1) * len, n_b, C, st);
      check_launch();
      std::vector<double> est;
      if (relres_of(res2, est)) {
        ++j;
        ++total;
        break;
      }
    }
    // x^ += Z y with H y = g (upper triangular, per column)
    std::vector<double> y((size_t)j * C, 0.0);
    for (int col = 0; col < C; ++col)
      for (int i = j - 1; i >= 0; --i) {
        double v = g[(size_t)i * C + col];
        for (int l = i + 1; l < j; ++l) v -= Hc[((size_t)i * m + l) * C + col] * y[(size_t)l * C + col];
        const double d = Hc[((size_t)i * m + i) * C + col];
        y[(size_t)i * C + col] = d != 0.0 ? v / d : 0.0;
      }
    if (j > 0) {
      to_dev(Hd.p, y.data(), (int64_t)j * C, st);
      launch_maxpy(Z.p, len, C, j, Hd.p, 1.0, xh, n_b, C, st);
      check_launch();
    }
  }
  if (D->singular) launch_sub_block0_mean(xh, n_b, nrhs, nb, D->sc_out.partials, D->sc_out.partial_cap, st);
  launch_transform_bwd(xh, VEC_F64, nrhs, D->perm, n_b, D->s, x_dev, ld, st);
  check_launch();
  CK(cudaStreamSynchronize(st));
  if (info) {
    info->iters = total;
    info->outer_iters = 0;
    info->converged = converged ? 1 : 0;
    if (info->relres) std::memcpy(info->relres, rel.data(), sizeof(double) * nrhs);
  }
  return converged ? AMGSYM_OK : AMGSYM_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// LRCFSAI(k) (Sec. 2.1, Thm. "correction", eqs. "Ydef", "LRC", "LRCFSAI"):
// the FSAI of A_inn, G_inn^T G_inn ~ A_inn^{-1}, corrected per block.  With
// X = G_inn A^_i G_inn^T (symmetric) and its k eigenpairs of the smallest
// eigenvalues (V_k, Lambda_k), Y = I - X has Sigma = I - Lambda and the
// correction is Z_k Theta_k Z_k^T with Z_k = G_inn^T V_k and
// Theta = Sigma (I - Sigma)^{-1}: Theta_t = (1 - lambda_t) / lambda_t.  The
// pairs come from Lanczos on X (Euclidean inner product, full
// reorthogonalisation) for all blocks at once; the preconditioner is
// symmetric, so the solve is PCG.

static void lrcfsai_setup(amgsym_t h, int32_t k, int32_t steps, uint64_t seed, cudaStream_t st) {
  Device* D = require_dev(h);
  D->lrcf_k = 0;
  D->lrcf_Z = D->lrcf_TZ = nullptr;
  D->lrcf_theta.clear();
  if (k == 0) return;
  const DevLevel& L = D->lv[0];
  if (L.cinv || !L.G.v64 || !L.Gt.v64)
    fail(AMGSYM_ERR_STATE, "LRCFSAI needs the FP64 FSAI factor of A_inn (a hierarchy of two levels or more, "
                           "opts.precisions with FP64)");
  const int32_t nb = D->nb, C = nb;
  const int64_t n_b = D->n_b, len = n_b * C;
  const int m = steps;
  ensure_work(D, 1, VEC_F64);
  Ctx c{D, C, VEC_F64, VAL_F64, false, st};
  PrecWork& W = D->w64;
  DevBuf Q((int64_t)(m + 1) * len), w(len), part((int64_t)mdot_blocks(n_b, C) * (m + 1) * C), Hd((int64_t)(m + 1) * C),
      sd(C);
  {
    std::vector<double> q0((size_t)len);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (auto& v : q0) v = U(rng);
    to_dev(Q.p, q0.data(), len, st);
  }
  std::vector<double> hh((size_t)(m + 1) * C), sv(C);
  auto normalise = [&](double* q) {  // q /= ||q|| per column; returns ||q||^2
    launch_mdot(q, 0, C, 1, q, n_b, C, part.p, Hd.p, st);
    check_launch();
    to_host(hh.data(), Hd.p, C, st);
    for (int j = 0; j < C; ++j) sv[j] = hh[j] > 0.0 ? 1.0 / std::sqrt(hh[j]) : 0.0;
    to_dev(sd.p, sv.data(), C, st);
    launch_colscale(q, sd.p, q, n_b, C, st);
    check_launch();
    return std::vector<double>(hh.begin(), hh.begin() + C);
  };
  auto apply_X = [&](const double* q, double* out) {  // out = G A^ G^T q
    spmm(c, L.Gt, VAL_F64, VEC_F64, VEC_F64, q, W.z, 1.0, 0.0, nullptr, false, nullptr);
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, W.z, W.q, 1.0, 0.0, nullptr, true, nullptr);
    spmm(c, L.G, VAL_F64, VEC_F64, VEC_F64, W.q, out, 1.0, 0.0, nullptr, false, nullptr);
  };
  normalise(Q.p);
  std::vector<double> alpha((size_t)m * C, 0.0), beta((size_t)m * C, 0.0);
  std::vector<int> mc(C, m);
  for (int j = 0; j < m; ++j) {
    apply_X(Q.p + (int64_t)j * len, w.p);
    std::vector<double> h_sum((size_t)(j + 1) * C, 0.0);
    for (int pass = 0; pass < 2; ++pass) {
      launch_mdot(Q.p, len, C, j + 1, w.p, n_b, C, part.p, Hd.p, st);
      launch_maxpy(Q.p, len, C, j + 1, Hd.p, -1.0, w.p, n_b, C, st);
      check_launch();
      to_host(hh.data(), Hd.p, (int64_t)(j + 1) * C, st);
      for (int64_t t = 0; t < (int64_t)(j + 1) * C; ++t) h_sum[t] += hh[t];
    }
    for (int col = 0; col < C; ++col) alpha[(size_t)j * C + col] = h_sum[(size_t)j * C + col];
    double* qn = Q.p + (int64_t)(j + 1) * len;
    CK(cudaMemcpyAsync(qn, w.p, sizeof(double) * (size_t)len, cudaMemcpyDeviceToDevice, st));
    const std::vector<double> b2 = normalise(qn);
    for (int col = 0; col < C; ++col) {
      double amax = 0.0;
      for (int i = 0; i <= j; ++i) amax = std::max(amax, std::fabs(alpha[(size_t)i * C + col]));
      const double b = b2[col] > 0.0 ? std::sqrt(b2[col]) : 0.0;
      beta[(size_t)j * C + col] = b;
      if (mc[col] == m && !(b > 1e-10 * amax)) mc[col] = j + 1;
    }
  }
  std::vector<double> theta((size_t)C * k, 0.0), Y((size_t)m * k * C, 0.0);
  std::vector<double> Th((size_t)k * C, 0.0);
  for (int col = 0; col < C; ++col) {
    const int mm = mc[col];
    std::vector<double> T((size_t)mm * mm, 0.0), V;
    for (int i = 0; i < mm; ++i) {
      T[(size_t)i * mm + i] = alpha[(size_t)i * C + col];
      if (i + 1 < mm) T[(size_t)i * mm + i + 1] = T[(size_t)(i + 1) * mm + i] = beta[(size_t)i * C + col];
    }
    jacobi_eig(T, V, mm);
    std::vector<int> order(mm);
    for (int i = 0; i < mm; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return T[(size_t)a * mm + a] < T[(size_t)b * mm + b]; });
    for (int t = 0; t < k && t < mm; ++t) {
      const int e = order[t];
      const double th = T[(size_t)e * mm + e];
      theta[(size_t)col * k + t] = th;
      Th[(size_t)t * C + col] = th > 0.0 ? (1.0 - th) / th : 0.0;  // Sigma (I - Sigma)^{-1}
      for (int i = 0; i < mm; ++i) Y[((size_t)t * m + i) * C + col] = V[(size_t)i * mm + e];
    }
  }
  // Z_t = G^T (Q Y_t), Theta Z_t
  double* Z = nullptr;
  double* TZ = nullptr;
  CK(cudaMalloc(&Z, sizeof(double) * (size_t)k * len));
  D->owned.push_back(Z);
  CK(cudaMalloc(&TZ, sizeof(double) * (size_t)k * len));
  D->owned.push_back(TZ);
  for (int t = 0; t < k; ++t) {
    CK(cudaMemsetAsync(w.p, 0, sizeof(double) * (size_t)len, st));
    to_dev(Hd.p, Y.data() + (size_t)t * m * C, (int64_t)m * C, st);
    launch_maxpy(Q.p, len, C, m, Hd.p, 1.0, w.p, n_b, C, st);
    spmm(c, L.Gt, VAL_F64, VEC_F64, VEC_F64, w.p, Z + (int64_t)t * len, 1.0, 0.0, nullptr, false, nullptr);
    to_dev(sd.p, Th.data() + (size_t)t * C, C, st);
    launch_colscale(Z + (int64_t)t * len, sd.p, TZ + (int64_t)t * len, n_b, C, st);
    check_launch();
  }
  CK(cudaStreamSynchronize(st));
  D->lrcf_k = k;
  D->lrcf_Z = Z;
  D->lrcf_TZ = TZ;
  D->lrcf_theta = theta;
}

// PCG on the reduced system with I (x) G_inn^T G_inn (+ the LRCFSAI correction),
// FP64, one CG per column (the preconditioner is block diagonal).
static amgsym_status fsai_pcg_impl(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                   const amgsym_solve_opts* sopts, int32_t use_lrc, cudaStream_t st,
                                   amgsym_solve_info* info) {
  Device* D = require_dev(h);
  amgsym_solve_opts o;
  amgsym_solve_opts_default(&o);
  if (sopts) o = *sopts;
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  if (ld < h->n || !b_dev || !x_dev) fail(AMGSYM_ERR_ARG, "bad vectors or ld");
  if (o.precision != AMGSYM_PREC_FP64) fail(AMGSYM_ERR_ARG, "the FSAI-preconditioned solve runs in FP64");
  if (!(o.tol > 0.0) || o.maxit < 1) fail(AMGSYM_ERR_ARG, "bad tolerance or maxit");
  const DevLevel& L = D->lv[0];
  if (L.cinv || !L.G.v64 || !L.Gt.v64) fail(AMGSYM_ERR_STATE, "no FP64 FSAI factor of A_inn");
  if (use_lrc && D->lrcf_k <= 0) fail(AMGSYM_ERR_STATE, "no LRCFSAI correction: call amgsym_lrcfsai_setup first");
  ensure_work(D, nrhs, VEC_F64);
  const int32_t nb = D->nb, C = nrhs * nb;
  const int64_t n_b = D->n_b, len = n_b * C;
  Ctx c{D, C, VEC_F64, VAL_F64, false, st};
  PrecWork& W = D->w64;  // r, z, p, q; x^ in D->xh
  DevBuf t(len), part((int64_t)mdot_blocks(n_b, C) * std::max(2, D->lrcf_k + 1) * C), Hd((int64_t)std::max(2, D->lrcf_k) * C),
      sd(C);
  double* bh = D->bh;
  double* xh = D->xh;
  launch_transform_fwd(b_dev, nrhs, ld, D->perm, n_b, D->s, bh, VEC_F64, st);
  check_launch();
  if (D->singular) launch_sub_block0_mean(bh, n_b, nrhs, nb, D->sc_out.partials, D->sc_out.partial_cap, st);
  if (o.use_x0)
    launch_transform_fwd(x_dev, nrhs, ld, D->perm, n_b, D->s, xh, VEC_F64, st);
  else
    CK(cudaMemsetAsync(xh, 0, sizeof(double) * (size_t)len, st));
  check_launch();
  double* r = static_cast<double*>(W.r);
  double* z = static_cast<double*>(W.z);
  double* p = static_cast<double*>(W.p);
  double* q = static_cast<double*>(W.q);
  std::vector<double> hv(C), bn2(nrhs, 0.0), rz(C), sv(C), ones(C, 1.0);
  auto coldot = [&](const double* a, const double* b, std::vector<double>& out) {
    launch_mdot(a, 0, C, 1, b, n_b, C, part.p, Hd.p, st);
    check_launch();
    to_host(out.data(), Hd.p, C, st);
  };
  auto precond = [&](const double* rr, double* zz) {  // zz = G^T G rr (+ Z Theta Z^T rr)
    spmm(c, L.G, VAL_F64, VEC_F64, VEC_F64, rr, t.p, 1.0, 0.0, nullptr, false, nullptr);
    spmm(c, L.Gt, VAL_F64, VEC_F64, VEC_F64, t.p, zz, 1.0, 0.0, nullptr, false, nullptr);
    if (use_lrc) {
      const int64_t vs = n_b * nb;
      launch_mdot(D->lrcf_TZ, vs, nb, D->lrcf_k, rr, n_b, C, part.p, Hd.p, st);
      launch_maxpy(D->lrcf_Z, vs, nb, D->lrcf_k, Hd.p, 1.0, zz, n_b, C, st);
      check_launch();
    }
  };
  auto relres = [&](const std::vector<double>& col2, std::vector<double>& rel) {
    rel.assign(nrhs, 0.0);
    for (int col = 0; col < C; ++col) rel[col / nb] += col2[col];
    bool ok = true;
    for (int rr = 0; rr < nrhs; ++rr) {
      rel[rr] = bn2[rr] > 0.0 ? std::sqrt(rel[rr] / bn2[rr]) : 0.0;
      if (!(rel[rr] <= o.tol)) ok = false;
    }
    return ok;
  };
  coldot(bh, bh, hv);
  for (int col = 0; col < C; ++col) bn2[col / nb] += hv[col];
  std::vector<double> rel;
  int it = 0;
  bool converged = false;
  for (int restart = 0; restart < 3 && !converged && it < o.maxit; ++restart) {
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, xh, r, -1.0, 1.0, bh, true, nullptr);  // r = b^ - A^ x^
    coldot(r, r, hv);
    if (relres(hv, rel)) {
      converged = true;
      break;
    }
    precond(r, z);
    CK(cudaMemcpyAsync(p, z, sizeof(double) * (size_t)len, cudaMemcpyDeviceToDevice, st));
    coldot(r, z, rz);
    for (; it < o.maxit; ++it) {
      spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, p, q, 1.0, 0.0, nullptr, true, nullptr);  // q = A^ p
      coldot(p, q, hv);
      for (int col = 0; col < C; ++col) sv[col] = hv[col] > 0.0 ? rz[col] / hv[col] : 0.0;  // alpha
      to_dev(Hd.p, sv.data(), C, st);
      launch_maxpy(p, 0, C, 1, Hd.p, 1.0, xh, n_b, C, st);   // x += alpha p
      launch_maxpy(q, 0, C, 1, Hd.p, -1.0, r, n_b, C, st);   // r -= alpha q
      check_launch();
      coldot(r, r, hv);
      if (relres(hv, rel)) {
        ++it;
        break;
      }
      precond(r, z);
      std::vector<double> rz_new(C);
      coldot(r, z, rz_new);
      for (int col = 0; col < C; ++col) sv[col] = rz[col] != 0.0 ? rz_new[col] / rz[col] : 0.0;  // beta
      rz = rz_new;
      to_dev(sd.p, sv.data(), C, st);
      launch_colscale(p, sd.p, p, n_b, C, st);                 // p = beta p
      to_dev(Hd.p, ones.data(), C, st);
      launch_maxpy(z, 0, C, 1, Hd.p, 1.0, p, n_b, C, st);      // p += z
      check_launch();
    }
    // confirm with the true residual
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, xh, r, -1.0, 1.0, bh, true, nullptr);
    coldot(r, r, hv);
    converged = relres(hv, rel);
  }
  if (D->singular) launch_sub_block0_mean(xh, n_b, nrhs, nb, D->sc_out.partials, D->sc_out.partial_cap, st);
  launch_transform_bwd(xh, VEC_F64, nrhs, D->perm, n_b, D->s, x_dev, ld, st);
  check_launch();
  CK(cudaStreamSynchronize(st));
  if (info) {
    info->iters = it;
    info->outer_iters = 0;
    info->converged = converged ? 1 : 0;
    if (info->relres) std::memcpy(info->relres, rel.data(), sizeof(double) * nrhs);
  }
  return converged ? AMGSYM_OK : AMGSYM_NOT_CONVERGED;
}

}  // namespace amgsym

using namespace amgsym;

extern "C" amgsym_status amgsym_lrc_setup(amgsym_t h, int32_t k, int32_t steps, uint64_t seed, void* stream) {
  try {
    if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
    if (k < 0 || k > 64) fail(AMGSYM_ERR_ARG, "k must be in [0, 64]");
    if (k > 0 && (steps < k || steps > 400)) fail(AMGSYM_ERR_ARG, "steps must be in [k, 400]");
    lrc_setup(h, k, steps, seed, static_cast<cudaStream_t>(stream));
    return AMGSYM_OK;
  } catch (const amgsym::Error& e) {
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}

extern "C" int32_t amgsym_lrc_values(amgsym_t h, double* theta) {
  if (!h || !h->dev) return -1;
  Device* D = h->dev;
  if (theta && D->lrc_k > 0) std::memcpy(theta, D->lrc_theta.data(), sizeof(double) * D->lrc_theta.size());
  return D->lrc_k;
}

extern "C" amgsym_status amgsym_solve_gmres(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                            const amgsym_solve_opts* sopts, int32_t restart, int32_t use_lrc,
                                            void* stream, amgsym_solve_info* info) {
  try {
    return gmres_impl(h, b_dev, x_dev, nrhs, ld, sopts, restart, use_lrc, static_cast<cudaStream_t>(stream), info);
  } catch (const amgsym::Error& e) {
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}

extern "C" amgsym_status amgsym_lrcfsai_setup(amgsym_t h, int32_t k, int32_t steps, uint64_t seed, void* stream) {
  try {
    if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
    if (k < 0 || k > 64) fail(AMGSYM_ERR_ARG, "k must be in [0, 64]");
    if (k > 0 && (steps < k || steps > 400)) fail(AMGSYM_ERR_ARG, "steps must be in [k, 400]");
    lrcfsai_setup(h, k, steps, seed, static_cast<cudaStream_t>(stream));
    return AMGSYM_OK;
  } catch (const amgsym::Error& e) {
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}

extern "C" int32_t amgsym_lrcfsai_values(amgsym_t h, double* theta) {
  if (!h || !h->dev) return -1;
  Device* D = h->dev;
  if (theta && D->lrcf_k > 0) std::memcpy(theta, D->lrcf_theta.data(), sizeof(double) * D->lrcf_theta.size());
  return D->lrcf_k;
}

extern "C" amgsym_status amgsym_solve_fsai(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                           const amgsym_solve_opts* sopts, int32_t use_lrc, void* stream,
                                           amgsym_solve_info* info) {
  try {
    return fsai_pcg_impl(h, b_dev, x_dev, nrhs, ld, sopts, use_lrc, static_cast<cudaStream_t>(stream), info);
  } catch (const amgsym::Error& e) {
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}
