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
// Lanczos in that inner product (thick-restarted, with deflated restarts that
// find every copy of a multiple eigenvalue: ritz_smallest) gives
// A^_i-orthonormal Ritz vectors u; then v = A^_i u is the left eigenvector
// that pairs with u (v^T X = lambda v^T, v^T u = 1).  Every block runs its own
// Lanczos as one column of the interleaved multi-column layout, so each step
// is one reduced SpMM and one V-cycle for all blocks at once.
//
// Application, per column of block i: z = w + U_i (Theta_i V_i^T w) with
// w = M_inn^{-1} r: k dots and k updates (k_krylov.cu).  The correction is not
// symmetric, hence GMRES (restarted, right-preconditioned, classical
// Gram-Schmidt with one reorthogonalisation) as in the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
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

// ---------------------------------------------------------------------------
// The k smallest eigenpairs of an operator X that is self-adjoint in the
// inner product <u, v> = u^T B v (B = A^_i for LRCAMG, B = I for LRCFSAI), for every column of the interleaved layout at
// once (column c is the problem of block c % nb).
//
// Lanczos with full reorthogonalisation (two classical Gram-Schmidt passes)
// keeps the whole projected matrix T = Q^T B X Q from the Gram-Schmidt
// coefficients, so the basis can be thick-restarted (Wu and Simon's
// thick-restart Lanczos, SIAM J. Matrix Anal. Appl. 22, 2000) from the `keep`
// Ritz vectors of the smallest Ritz values and the last Lanczos vector
// whenever it reaches W vectors, without any special form of T.  A run ends
// when the k smallest Ritz pairs and a buffer of max(4, k / 2) more have
// residuals ||X u - theta u||_B <= tol * theta (|beta_W y_W| per pair).  One Krylov sequence holds a single
// copy of a multiple eigenvalue (the mirror blocks of a cube have 3-fold
// ones, and a correction that misses the copies barely helps), so the search
// restarts from new random vectors kept B-orthogonal to every pair found so
// far (deflation by locking) and stops when a run finds nothing below the
// k-th smallest value found before.  The pairs kept are the k smallest of all
// runs.  Ritz values at rounding level relative to the largest (a null
// space) are never kept.
constexpr int kRitzMaxRuns = 4;
constexpr int kRitzMaxCycles = 200;

struct RitzOp {
  bool b_inner = false;                                                       // B-inner product, else Euclidean
  std::function<void(const double* q, const double* bq, double* out)> apply;  // out = X q (bq = B q)
  std::function<void(const double* q, double* out)> bmul;                     // out = B q
  // optional: picks a representative of q modulo the null space of a
  // semi-definite B (in place), before B q and the normalisation
  std::function<void(double* q)> project;
};

// Eigenpairs of the leading m x m part of a column's projected matrix,
// ascending, without the rounding-level ones.
struct ColRitz {
  int m = 0;
  std::vector<double> th, Y;  // th[e], Y[i * m + e]
  std::vector<int> order;     // all values ascending
  std::vector<int> usable;    // ascending, rounding-level ones left out
};

ColRitz col_ritz(const std::vector<double>& T, int W, int col, int m) {
  ColRitz r;
  r.m = m;
  if (m == 0) return r;
  std::vector<double> A((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = T[((size_t)col * W + i) * W + j];
  jacobi_eig(A, r.Y, m);
  r.th.resize(m);
  for (int e = 0; e < m; ++e) r.th[e] = A[(size_t)e * m + e];
  r.order.resize(m);
  for (int e = 0; e < m; ++e) r.order[e] = e;
  std::sort(r.order.begin(), r.order.end(), [&](int a, int b) { return r.th[a] < r.th[b]; });
  double top = 0.0;
  for (double v : r.th) top = std::max(top, std::fabs(v));
  for (int e : r.order)
    if (r.th[e] > 1e-10 * top) r.usable.push_back(e);
  return r;
}

// U (and BU = B U when op.b_inner): k vectors of n_b x C; vector t holds in
// column c the t-th smallest pair of column c (zero where the column has
// fewer), theta[c * k + t] its Ritz value (0 where none).  lock0: n0
// B-orthonormal vectors (B lock0 = lock0b) every pair stays B-orthogonal to.
void ritz_smallest(const Ctx& c, const RitzOp& op, int k, int W, double tol, uint64_t seed, const double* lock0,
                   const double* lock0b, int n0, double* U, double* BU, std::vector<double>& theta) {
  Device* D = c.D;
  cudaStream_t st = c.st;
  const int32_t C = c.C;
  const int64_t n_b = D->n_b, len = n_b * C;
  const bool bi = op.b_inner;
  const int keep = std::min(W - 2, std::max(k + 4, W / 2));
  // pairs a run must converge: k and a buffer (max(4, k / 2)), so that an
  // eigenvalue below the k-th one the basis has barely seen yet is not
  // skipped when the first k pairs meet a rough tolerance
  const int kc = std::max(k, std::min(keep - 1, k + std::max(4, k / 2)));
  const int pcap = kRitzMaxRuns * k;
  const int jmax = std::max(std::max(W + 1, pcap), std::max(n0, 1));
  DevBuf QA((int64_t)(W + 1) * len), QB((int64_t)(W + 1) * len), BQA(bi ? (int64_t)(W + 1) * len : 0),
      BQB(bi ? (int64_t)(W + 1) * len : 0), pool((int64_t)pcap * len), bpool(bi ? (int64_t)pcap * len : 0), w(len),
      bw(bi ? len : 0), part((int64_t)mdot_blocks(n_b, C) * jmax * C), Hd((int64_t)2 * (W + 1) * C),
      Hl((int64_t)jmax * C), Hc((int64_t)std::max(keep, k) * jmax * C), sd(C);
  double* qa = QA.p;
  double* qb = QB.p;
  double* bqa = bi ? BQA.p : QA.p;
  double* bqb = bi ? BQB.p : QB.p;
  double* bp = bi ? bpool.p : pool.p;
  double* bwp = bi ? bw.p : w.p;
  std::vector<double> hh((size_t)2 * (W + 1) * C), sv(C), b2(C);
  std::vector<double> pool_theta((size_t)pcap * C, HUGE_VAL);
  int P = 0;

  // w -= V (BV^T w) for a B-orthonormal set of J vectors
  auto orth_set = [&](const double* V, const double* BV, int J) {
    if (J <= 0) return;
    launch_mdot(BV, len, C, J, w.p, n_b, C, part.p, Hl.p, st);
    launch_maxpy(V, len, C, J, Hl.p, -1.0, w.p, n_b, C, st);
  };
  auto norm2 = [&]() {  // b2 = w^T B w per column (bw = B w)
    if (bi) op.bmul(w.p, bw.p);
    launch_mdot(w.p, 0, C, 1, bwp, n_b, C, part.p, Hl.p, st);
    check_launch();
    to_host(b2.data(), Hl.p, C, st);
  };
  auto put_scaled = [&](double* q, double* bq) {  // q = w * sv, bq = B w * sv
    to_dev(sd.p, sv.data(), C, st);
    launch_colscale(w.p, sd.p, q, n_b, C, st);
    if (bi) launch_colscale(bw.p, sd.p, bq, n_b, C, st);
    check_launch();
  };
  // dst_t = sum_j src_j coef[t][j][c], t < nt (coef [nt][J][C], uploaded)
  auto combine = [&](const double* src, int J, const std::vector<double>& coef, int nt, double* dst) {
    to_dev(Hc.p, coef.data(), (int64_t)nt * J * C, st);
    for (int t = 0; t < nt; ++t) {
      CK(cudaMemsetAsync(dst + (int64_t)t * len, 0, sizeof(double) * (size_t)len, st));
      launch_maxpy(src, len, C, J, Hc.p + (int64_t)t * J * C, 1.0, dst + (int64_t)t * len, n_b, C, st);
    }
    check_launch();
  };

  for (int run = 0; run < kRitzMaxRuns; ++run) {
    // start vector: uniform[-1, 1], B-orthogonal to the locked vectors
    {
      std::vector<double> q0((size_t)len);
      std::mt19937_64 rng(seed + 0x9E3779B97F4A7C15ull * (uint64_t)run);
      std::uniform_real_distribution<double> Ud(-1.0, 1.0);
      for (auto& v : q0) v = Ud(rng);
      to_dev(w.p, q0.data(), len, st);
    }
    if (op.project) op.project(w.p);
    norm2();
    const std::vector<double> b2_start = b2;
    for (int pass = 0; pass < 2; ++pass) {
      orth_set(lock0, lock0b, n0);
      orth_set(pool.p, bp, P);
    }
    check_launch();
    if (op.project) op.project(w.p);
    norm2();
    std::vector<char> open(C, 0);
    bool any_open = false;
    for (int col = 0; col < C; ++col) {
      open[col] = b2[col] > 1e-20 * b2_start[col];  // else the locked vectors span the column's space
      sv[col] = open[col] ? 1.0 / std::sqrt(b2[col]) : 0.0;
      any_open = any_open || open[col];
    }
    if (!any_open) break;
    put_scaled(qa, bqa);
    std::vector<double> T((size_t)C * W * W, 0.0), beta(C, 0.0), tscale(C, 0.0);
    std::vector<int> valid(C, 0);
    std::vector<ColRitz> rz(C);
    int nk = 0;
    for (int cycle = 0;; ++cycle) {
      for (int j = nk; j < W; ++j) {
        op.apply(qa + (int64_t)j * len, bqa + (int64_t)j * len, w.p);
        for (int pass = 0; pass < 2; ++pass) {
          orth_set(lock0, lock0b, n0);
          orth_set(pool.p, bp, P);
          double* hp = Hd.p + (int64_t)pass * (W + 1) * C;
          launch_mdot(bqa, len, C, j + 1, w.p, n_b, C, part.p, hp, st);
          launch_maxpy(qa, len, C, j + 1, hp, -1.0, w.p, n_b, C, st);
        }
        check_launch();
        to_host(hh.data(), Hd.p, (int64_t)2 * (W + 1) * C, st);
        if (op.project) op.project(w.p);
        norm2();
        for (int col = 0; col < C; ++col) {
          sv[col] = 0.0;
          if (!open[col]) continue;
          for (int i = 0; i <= j; ++i) {
            const double t = hh[(size_t)i * C + col] + hh[(size_t)(W + 1 + i) * C + col];
            T[((size_t)col * W + i) * W + j] = T[((size_t)col * W + j) * W + i] = t;
            tscale[col] = std::max(tscale[col], std::fabs(t));
          }
          valid[col] = j + 1;
          const double b = std::sqrt(std::max(b2[col], 0.0));
          if (b > 1e-10 * tscale[col]) {
            beta[col] = b;
            sv[col] = 1.0 / b;
          } else {  // invariant subspace: the column's Ritz pairs are exact
            beta[col] = 0.0;
            open[col] = 0;
          }
        }
        put_scaled(qa + (int64_t)(j + 1) * len, bqa + (int64_t)(j + 1) * len);
      }
      bool conv = true;
      for (int col = 0; col < C; ++col) {
        rz[col] = col_ritz(T, W, col, valid[col]);
        const ColRitz& r = rz[col];
        const int nk_c = std::min<int>(kc, (int)r.usable.size());
        for (int t = 0; t < nk_c && open[col]; ++t) {
          const int e = r.usable[t];
          if (!(std::fabs(beta[col] * r.Y[(size_t)(r.m - 1) * r.m + e]) <= tol * std::fabs(r.th[e]))) conv = false;
        }
      }
      if (conv || cycle + 1 >= kRitzMaxCycles) break;
      // thick restart: the keep smallest Ritz vectors, then the last Lanczos vector
      std::vector<double> coef((size_t)keep * W * C, 0.0);
      for (int col = 0; col < C; ++col) {
        const ColRitz& r = rz[col];
        for (int t = 0; t < keep && t < r.m; ++t)
          for (int i = 0; i < r.m; ++i) coef[((size_t)t * W + i) * C + col] = r.Y[(size_t)i * r.m + r.order[t]];
      }
      combine(qa, W, coef, keep, qb);
      if (bi) combine(bqa, W, coef, keep, bqb);
      CK(cudaMemcpyAsync(qb + (int64_t)keep * len, qa + (int64_t)W * len, sizeof(double) * (size_t)len,
                         cudaMemcpyDeviceToDevice, st));
      if (bi)
        CK(cudaMemcpyAsync(bqb + (int64_t)keep * len, bqa + (int64_t)W * len, sizeof(double) * (size_t)len,
                           cudaMemcpyDeviceToDevice, st));
      std::swap(qa, qb);
      std::swap(bqa, bqb);
      std::fill(T.begin(), T.end(), 0.0);
      for (int col = 0; col < C; ++col) {
        const ColRitz& r = rz[col];
        valid[col] = std::min(keep, r.m);
        tscale[col] = 0.0;
        for (int t = 0; t < valid[col]; ++t) {
          const double th = r.th[r.order[t]];
          T[((size_t)col * W + t) * W + t] = th;
          tscale[col] = std::max(tscale[col], std::fabs(th));
        }
      }
      nk = keep;
    }
    // the run's k smallest pairs join the locked pool
    std::vector<double> coef((size_t)k * W * C, 0.0);
    bool any_new = false;
    for (int col = 0; col < C; ++col) {
      const ColRitz& r = rz[col];
      std::vector<double> prev;
      for (int p = 0; p < P; ++p)
        if (pool_theta[(size_t)p * C + col] < HUGE_VAL) prev.push_back(pool_theta[(size_t)p * C + col]);
      std::sort(prev.begin(), prev.end());
      const double kth = (int)prev.size() >= k ? prev[k - 1] : HUGE_VAL;
      for (int t = 0; t < k && t < (int)r.usable.size(); ++t) {
        const int e = r.usable[t];
        for (int i = 0; i < r.m; ++i) coef[((size_t)t * W + i) * C + col] = r.Y[(size_t)i * r.m + e];
        pool_theta[(size_t)(P + t) * C + col] = r.th[e];
        if (r.th[e] < kth) any_new = true;
      }
    }
    combine(qa, W, coef, k, pool.p + (int64_t)P * len);
    if (bi) combine(bqa, W, coef, k, bpool.p + (int64_t)P * len);
    P += k;
    if (!any_new) break;
  }
  // the k smallest of every run, gathered per column
  theta.assign((size_t)C * k, 0.0);
  std::vector<double> sel((size_t)k * std::max(P, 1) * C, 0.0);
  for (int col = 0; col < C; ++col) {
    std::vector<int> idx;
    for (int p = 0; p < P; ++p)
      if (pool_theta[(size_t)p * C + col] < HUGE_VAL) idx.push_back(p);
    std::sort(idx.begin(), idx.end(),
              [&](int a, int b) { return pool_theta[(size_t)a * C + col] < pool_theta[(size_t)b * C + col]; });
    for (int t = 0; t < k && t < (int)idx.size(); ++t) {
      sel[((size_t)t * P + idx[t]) * C + col] = 1.0;
      theta[(size_t)col * k + t] = pool_theta[(size_t)idx[t] * C + col];
    }
  }
  if (P > 0) {
    combine(pool.p, P, sel, k, U);
    if (bi) combine(bpool.p, P, sel, k, BU);
  } else {
    CK(cudaMemsetAsync(U, 0, sizeof(double) * (size_t)k * len, st));
    if (bi) CK(cudaMemsetAsync(BU, 0, sizeof(double) * (size_t)k * len, st));
  }
  CK(cudaStreamSynchronize(st));
}

}  // namespace

// LRCAMG(k) setup: X = M_inn^{-1} A^_i is self-adjoint in the A^_i inner
// product; its k smallest eigenpairs per block give U (A^_i-orthonormal) and
// V_t = Theta_t A^_i u_t.
static void lrc_setup(amgsym_t h, int32_t k, int32_t steps, double tol, uint64_t seed, cudaStream_t st) {
  Device* D = require_dev(h);
  D->lrc_k = 0;
  D->lrc_U = D->lrc_V = nullptr;  // the old arrays stay owned until device_free
  D->lrc_theta.clear();
  if (k == 0) return;
  const int32_t C = D->nb;
  const int64_t n_b = D->n_b, len = n_b * C;
  ensure_work(D, 1, VEC_F64);
  Ctx c{D, C, VEC_F64, VAL_F64, false, st};
  c.fuse = true;
  RitzOp op;
  op.b_inner = true;
  op.bmul = [&](const double* q, double* out) {
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, q, out, 1.0, 0.0, nullptr, true, nullptr);
  };
  op.apply = [&](const double*, const double* bq, double* out) {  // M_inn^{-1} (A^ q)
    vcycle_apply(c, bq, out);
    check_launch();
  };
  if (D->singular) {
    // A^_0 is semi-definite (A^_0 1 = 0): its inner product does not see the
    // constant, which rounding would let grow into spurious small Ritz
    // values; vectors are kept with zero mean in block 0 (the same classes)
    op.project = [&](double* q) {
      launch_sub_block0_mean(q, n_b, 1, C, D->sc_out.partials, D->sc_out.partial_cap, st);
      check_launch();
    };
  }
  double* U = nullptr;
  double* Vv = nullptr;
  CK(cudaMalloc(&U, sizeof(double) * (size_t)k * len));
  D->owned.push_back(U);
  CK(cudaMalloc(&Vv, sizeof(double) * (size_t)k * len));
  D->owned.push_back(Vv);
  std::vector<double> theta;
  ritz_smallest(c, op, k, steps, tol, seed, nullptr, nullptr, 0, U, Vv, theta);
  // V_t = Theta_t A^ u_t with Theta_t = (1 - lambda_t) / lambda_t (eq. "LRC_AMG")
  DevBuf sd(C);
  std::vector<double> th(C);
  for (int t = 0; t < k; ++t) {
    for (int col = 0; col < C; ++col) {
      const double l = theta[(size_t)col * k + t];
      th[col] = l > 0.0 ? (1.0 - l) / l : 0.0;
    }
    to_dev(sd.p, th.data(), C, st);
    launch_colscale(Vv + (int64_t)t * len, sd.p, Vv + (int64_t)t * len, n_b, C, st);
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
// pairs come from the restarted Lanczos of ritz_smallest on X (Euclidean inner
// product) for all blocks at once; the preconditioner is symmetric, so the
// solve is PCG.

static void lrcfsai_setup(amgsym_t h, int32_t k, int32_t steps, double tol, uint64_t seed, cudaStream_t st) {
  Device* D = require_dev(h);
  D->lrcf_k = 0;
  D->lrcf_Z = D->lrcf_TZ = nullptr;
  D->lrcf_theta.clear();
  if (k == 0) return;
  const DevLevel& L = D->lv[0];
  if (L.cinv || !L.G.v64 || !L.Gt.v64)
    fail(AMGSYM_ERR_STATE, "LRCFSAI needs the FP64 FSAI factor of A_inn (a hierarchy of two levels or more, "
                           "opts.precisions with FP64)");
  const int32_t C = D->nb;
  const int64_t n_b = D->n_b, len = n_b * C;
  ensure_work(D, 1, VEC_F64);
  Ctx c{D, C, VEC_F64, VAL_F64, false, st};
  PrecWork& W = D->w64;
  RitzOp op;
  op.apply = [&](const double* q, const double*, double* out) {  // G A^ G^T q
    spmm(c, L.Gt, VAL_F64, VEC_F64, VEC_F64, q, W.z, 1.0, 0.0, nullptr, false, nullptr);
    spmm(c, D->Ainn, VAL_F64, VEC_F64, VEC_F64, W.z, W.q, 1.0, 0.0, nullptr, true, nullptr);
    spmm(c, L.G, VAL_F64, VEC_F64, VEC_F64, W.q, out, 1.0, 0.0, nullptr, false, nullptr);
  };
  // A singular block 0 (A^_0 1 = 0) gives X the null vector G^{-T} 1, found
  // by back substitution with the lower-triangular host factor; the pairs stay
  // orthogonal to it.
  DevBuf nullv(D->singular ? len : 0);
  if (D->singular) {
    const Csr& G = h->H.levels[0].G;
    std::vector<double> r((size_t)n_b, 1.0), v((size_t)n_b, 0.0);
    for (int64_t i = n_b - 1; i >= 0; --i) {
      double d = 0.0;
      for (int64_t e = G.ptr[i]; e < G.ptr[i + 1]; ++e)
        if (G.idx[e] == i) d = G.val[e];
      if (!(d != 0.0)) fail(AMGSYM_ERR_STATE, "FSAI factor with a zero diagonal");
      v[i] = r[i] / d;
      for (int64_t e = G.ptr[i]; e < G.ptr[i + 1]; ++e)
        if (G.idx[e] < i) r[G.idx[e]] -= G.val[e] * v[i];
    }
    double nv = 0.0;
    for (double x : v) nv += x * x;
    nv = std::sqrt(nv);
    std::vector<double> hv((size_t)len, 0.0);
    for (int64_t i = 0; i < n_b; ++i) hv[(size_t)i * C] = v[i] / nv;  // column 0: block 0
    to_dev(nullv.p, hv.data(), len, st);
  }
  DevBuf Uu((int64_t)k * len), sd(C);
  std::vector<double> theta;
  ritz_smallest(c, op, k, steps, tol, seed, nullv.p, nullv.p, D->singular ? 1 : 0, Uu.p, nullptr, theta);
  // Z_t = G^T u_t and Theta_t Z_t, Theta_t = (1 - lambda_t) / lambda_t
  double* Z = nullptr;
  double* TZ = nullptr;
  CK(cudaMalloc(&Z, sizeof(double) * (size_t)k * len));
  D->owned.push_back(Z);
  CK(cudaMalloc(&TZ, sizeof(double) * (size_t)k * len));
  D->owned.push_back(TZ);
  std::vector<double> th(C);
  for (int t = 0; t < k; ++t) {
    spmm(c, L.Gt, VAL_F64, VEC_F64, VEC_F64, Uu.p + (int64_t)t * len, Z + (int64_t)t * len, 1.0, 0.0, nullptr, false,
         nullptr);
    for (int col = 0; col < C; ++col) {
      const double l = theta[(size_t)col * k + t];
      th[col] = l > 0.0 ? (1.0 - l) / l : 0.0;  // Sigma (I - Sigma)^{-1}
    }
    to_dev(sd.p, th.data(), C, st);
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

extern "C" amgsym_status amgsym_lrc_setup(amgsym_t h, int32_t k, int32_t steps, double tol, uint64_t seed,
                                          void* stream) {
  try {
    if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
    if (k < 0 || k > 64) fail(AMGSYM_ERR_ARG, "k must be in [0, 64]");
    if (k > 0 && (steps < k + 2 || steps > 400)) fail(AMGSYM_ERR_ARG, "steps must be in [k + 2, 400]");
    if (k > 0 && !(tol > 0.0 && tol <= 1.0)) fail(AMGSYM_ERR_ARG, "tol must be in (0, 1]");
    lrc_setup(h, k, steps, tol, seed, static_cast<cudaStream_t>(stream));
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

extern "C" amgsym_status amgsym_lrcfsai_setup(amgsym_t h, int32_t k, int32_t steps, double tol, uint64_t seed,
                                              void* stream) {
  try {
    if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
    if (k < 0 || k > 64) fail(AMGSYM_ERR_ARG, "k must be in [0, 64]");
    if (k > 0 && (steps < k + 2 || steps > 400)) fail(AMGSYM_ERR_ARG, "steps must be in [k + 2, 400]");
    if (k > 0 && !(tol > 0.0 && tol <= 1.0)) fail(AMGSYM_ERR_ARG, "tol must be in (0, 1]");
    lrcfsai_setup(h, k, steps, tol, seed, static_cast<cudaStream_t>(stream));
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
