// Device residency of a problem and the solve of Alg. 1 ("symsolver"):
// forward transform, 2^s decoupled PCG solves run as one multi-column PCG
// preconditioned by I (x) M_inn^{-1} (eqs. "AMGinn", "LRCAMG" with k = 0),
// backward transform.  Optional FP64 iterative refinement around an FP32
// inner PCG (mixed precision).  Every arithmetic step runs in the kernels of
// k_spmm.cu / k_misc.cu; this file only allocates, uploads and sequences.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <random>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <vector>

#include "device.h"
#include "internal.h"
#include "solver.h"

namespace amgsym {

uint64_t next_generation() {
  static std::atomic<uint64_t> counter{0};
  return ++counter;
}

void check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fail(AMGSYM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Per-launch timing hooks (see Profiler in solver.h).

thread_local Profiler* t_prof = nullptr;

ProfScope::ProfScope(cudaStream_t st) : st_(st) {
  if (!t_prof) return;
  CK(cudaEventCreate(&ev0_));
  CK(cudaEventRecord(ev0_, st_));
}

ProfScope::~ProfScope() {
  if (ev0_) cudaEventDestroy(ev0_);  // not ended (an error unwound the launch)
}

void ProfScope::end(const std::string& kernel, const std::string& role, int level, int64_t bytes) {
  if (!ev0_ || !t_prof) return;
  ProfRecord r;
  r.kernel = kernel;
  r.role = role;
  r.level = level;
  r.phase = t_prof->phase;
  r.bytes = bytes;
  r.e0 = ev0_;
  ev0_ = nullptr;
  CK(cudaEventCreate(&r.e1));
  CK(cudaEventRecord(r.e1, st_));
  t_prof->recs.push_back(r);
}

static const char* tname(ValType t) { return t == VAL_F64 ? "double" : t == VAL_F32 ? "float" : "bf16"; }
static const char* tname(VecType t) { return t == VEC_F64 ? "double" : "float"; }
static int64_t vsize(ValType t) { return t == VAL_F64 ? 8 : t == VAL_F32 ? 4 : 2; }
static int64_t xsize(VecType t) { return t == VEC_F64 ? 8 : 4; }

// Which level matrix M is ("A", "P", "R", "G", "Gt") and its level.
static std::string matrix_name(const Device* D, const DevCsr& M, int* level) {
  for (size_t l = 0; l < D->lv.size(); ++l) {
    const DevLevel& L = D->lv[l];
    *level = (int)l;
    if (M.idx == L.A.idx) return "A";
    if (M.idx == L.P.idx) return "P";
    if (M.idx == L.R.idx) return "R";
    if (M.idx == L.G.idx) return "G";
    if (M.idx == L.Gt.idx) return "Gt";
  }
  *level = 0;
  if (D->has_amgr) {
    if (M.idx == D->amgr.Pb.idx) return "AMGR P_b";
    if (M.idx == D->amgr.Rb.idx) return "AMGR R_b";
    if (M.idx == D->amgr.GK.idx) return "AMGR G_K";
    if (M.idx == D->amgr.GKt.idx) return "AMGR G_K^T";
  }
  *level = -1;
  return "?";
}

// Algorithmic bytes of one SpMM launch: the matrix (stored diagonals, or CSR
// values + column indices + row pointers), X once, Y once, each epilogue
// operand once (an operand that is X itself is not counted twice), the
// diagonal-smoother vectors and the interface lookups.
static int64_t spmm_bytes(const Device* D, const DevCsr& M, ValType mt, VecType xt, VecType ot, const SpmmArgs& a) {
  const int64_t rows = a.rows, C = a.C;
  int64_t b = 0;
  if (a.ndiag > 0) {
    int nstored = 0;
    for (int d = 0; d < a.ndiag; ++d) nstored = std::max(nstored, a.dsrc[d] + 1);
    b += (int64_t)nstored * rows * vsize(mt);
  } else if (spmm_uses_halo(xt, a)) {
    // values, 16-bit local columns, row pointers, tile halo pointers and lists
    b += M.nnz * (vsize(mt) + 2) + 4 * (rows + 1) + 4 * ((int64_t)M.htiles + 1) + 4 * M.hsum;
  } else {
    b += M.nnz * (vsize(mt) + 4) + 4 * (rows + 1);
  }
  std::set<const void*> seen;
  auto rd = [&](const void* p, int64_t n) {
    if (p && seen.insert(p).second) b += n;
  };
  rd(a.X, C * xsize(xt) * (int64_t)M.cols);
  b += C * xsize(ot) * rows;
  if (a.beta != 0.0) rd(a.Z, C * xsize(xt) * rows);
  if (a.dot.mode == DOT_WY) rd(a.dot.W, C * xsize(xt) * rows);
  if (a.jmode) rd(a.jd, xsize(xt) * rows);
  if (a.jmode == 1) b += C * xsize(ot) * rows;
  if (a.imask) {
    const int64_t words = (rows + 31) / 32;
    const bool f64 = (mt == VAL_F64) || (xt == VEC_F64);
    b += words * 8 + ((int64_t)a.nflag + 1) * 4 + (int64_t)a.nflag * 4 +
         D->iface.n_entries * (4 + (int64_t)a.nb * (f64 ? 8 : 4));
  }
  return b;
}

static void run_spmm(const Ctx& c, const DevCsr& M, ValType mt, VecType xt, VecType ot, const SpmmArgs& a) {
  ProfScope ps(c.st);
  launch_spmm(mt, xt, ot, a, c.st);
  check_launch();
  if (!ps.on()) return;
  int cpt = 0, kl = 0;
  spmm_resolved_tile(xt, ot, a, &cpt, &kl);
  const bool dot = a.dot.mode != DOT_NONE, ifc = a.imask != nullptr, dia = a.ndiag > 0;
  const char* kname = spmm_uses_stencil(mt, xt, ot, a) ? "stencil_kernel<"
                      : spmm_uses_halo(xt, a)                ? "spmm_halo_kernel<"
                      : spmm_uses_sell(xt, ot, a)            ? "sell_kernel<"
                                                             : "spmm_kernel<";
  const std::string kernel = std::string(kname) + tname(mt) + "," + tname(xt) + "," + tname(ot) + "," +
                             std::to_string(cpt) + "," + std::to_string(kl) + "," + (dot ? "1" : "0") + "," +
                             (ifc ? "1" : "0") + "," + (dia ? "1" : "0") + ">";
  int level = -1;
  std::string role;
  if (ifc && c.D->symc && M.idx == c.D->symc->inn.idx) {
    role = "AMGR A_c in the transformed basis";
    level = 0;
  } else if (ifc) {
    role = xt == VEC_F64 && ot == VEC_F32 ? "FP64 outer residual b^ - A^ x^" : "reduced SpMM A^ p";
    level = -1;
  } else {
    const std::string m = matrix_name(c.D, M, &level);
    role = "L" + std::to_string(level) + " " + m;
    if (a.jmode == 1)
      role += " restrict + next-level presmooth";
    else if (a.jmode == 2)
      role += " residual + postsmooth";
    else if (a.beta != 0.0 && a.alpha == -1.0)
      role += " residual";
    else if (a.beta != 0.0)
      role += " update";
  }
  if (dot) role += a.dot.mode == DOT_WY ? " + <w,y>" : " + <y,y>";
  ps.end(kernel, role, level, spmm_bytes(c.D, M, mt, xt, ot, a));
}

template <typename T>
static T* dalloc(std::vector<void*>& owner, int64_t count) {
  if (count <= 0) return nullptr;
  void* p = nullptr;
  CK(cudaMalloc(&p, sizeof(T) * (size_t)count));
  owner.push_back(p);
  return static_cast<T*>(p);
}

template <typename T>
static T* upload(std::vector<void*>& owner, const T* src, int64_t count) {
  T* d = dalloc<T>(owner, count);
  if (count > 0) CK(cudaMemcpy(d, src, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice));
  return d;
}

// Halo tiles of a CSR matrix (the halo-staged product, see DevCsr): the
// largest tile height of 256, 128, 64 or 32 rows whose largest halo (distinct
// columns of a tile) takes at most budget_bytes at 32 bytes per X row (8 FP32
// columns) and fits 16-bit local indices.  False if none does.
struct HostHalo {
  int32_t rows = 0, hmax = 0;
  std::vector<int32_t> hptr, hx;
  std::vector<uint16_t> lidx;
};

static bool build_halo(const Csr& M, int64_t budget_bytes, HostHalo& H) {
  const int64_t n = M.rows;
  if (n <= 0 || M.nnz() == 0 || budget_bytes <= 0) return false;
  for (int R : {256, 128, 64, 32}) {
    const int64_t nt = (n + R - 1) / R;
    std::vector<int32_t> size((size_t)nt);
    int32_t hmax = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : hmax)
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t kb = M.ptr[t * R], ke = M.ptr[std::min(n, (t + 1) * R)];
      std::vector<int32_t> c(M.idx.begin() + kb, M.idx.begin() + ke);
      std::sort(c.begin(), c.end());
      size[t] = (int32_t)(std::unique(c.begin(), c.end()) - c.begin());
      hmax = std::max(hmax, size[t]);
    }
    if ((int64_t)hmax * 32 > budget_bytes || hmax > 65535) continue;
    H.rows = R;
    H.hmax = hmax;
    H.hptr.assign((size_t)nt + 1, 0);
    for (int64_t t = 0; t < nt; ++t) H.hptr[t + 1] = H.hptr[t] + size[t];
    H.hx.resize((size_t)H.hptr[nt]);
    H.lidx.resize((size_t)M.nnz());
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t kb = M.ptr[t * R], ke = M.ptr[std::min(n, (t + 1) * R)];
      int32_t* h = H.hx.data() + H.hptr[t];
      std::vector<int32_t> c(M.idx.begin() + kb, M.idx.begin() + ke);
      std::sort(c.begin(), c.end());
      std::copy(c.begin(), std::unique(c.begin(), c.end()), h);
      for (int64_t k = kb; k < ke; ++k)
        H.lidx[k] = (uint16_t)(std::lower_bound(h, h + size[t], M.idx[k]) - h);
    }
    return true;
  }
  return false;
}

// Interface couplings (entries sorted by (row, column), values [entry][block])
// in the per-row flag form the SpMM looks up (see DevIface).
static DevIface upload_iface(std::vector<void*>& owner, int64_t rows, const std::vector<int32_t>& irow,
                             const std::vector<int32_t>& icol, const std::vector<double>& ivals, int32_t nb) {
  DevIface F;
  const int64_t ne = (int64_t)irow.size();
  if (ne <= 0) return F;
  const int64_t words = (rows + 31) / 32;
  std::vector<uint32_t> mask(words, 0);
  std::vector<int32_t> prefix(words, 0), iptr, irows;
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t r = irow[e];
    if (e == 0 || irow[e - 1] != r) {
      mask[r >> 5] |= 1u << (r & 31);
      iptr.push_back((int32_t)e);
      irows.push_back(r);
    }
  }
  iptr.push_back((int32_t)ne);
  int32_t run = 0;
  for (int64_t w = 0; w < words; ++w) {
    prefix[w] = run;
    run += __builtin_popcount(mask[w]);
  }
  F.n_rows_flagged = run;
  F.n_entries = ne;
  F.mask = upload(owner, mask.data(), words);
  F.prefix = upload(owner, prefix.data(), words);
  F.iptr = upload(owner, iptr.data(), (int64_t)iptr.size());
  F.irows = upload(owner, irows.data(), (int64_t)irows.size());
  F.icol = upload(owner, icol.data(), ne);
  F.ival64 = upload(owner, ivals.data(), ne * nb);
  std::vector<float> v32(ivals.begin(), ivals.end());
  F.ival32 = upload(owner, v32.data(), ne * nb);
  return F;
}

// Sliced form (SELL-32) of a CSR matrix, see DevCsr: rows sorted by length
// (longest first, stable) within windows of kSellWindow rows, then cut into
// slices of 32; false when the padded entries would not fit 32-bit offsets.
struct HostSell {
  std::vector<int32_t> sptr, srow, sidx;
  std::vector<int64_t> src;  // CSR entry of each slot, -1 for padding
};

static bool build_sell(const Csr& M, HostSell& S) {
  const int64_t n = M.rows;
  if (n <= 0) return false;
  std::vector<int32_t> order((size_t)n);
  for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  auto len = [&](int32_t r) { return M.ptr[r + 1] - M.ptr[r]; };
  for (int64_t w0 = 0; w0 < n; w0 += kSellWindow) {
    const int64_t w1 = std::min<int64_t>(n, w0 + kSellWindow);
    std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int32_t a, int32_t b) { return len(a) > len(b); });
  }
  const int64_t ns = (n + 31) / 32;
  S.sptr.assign((size_t)ns + 1, 0);
  S.srow.assign((size_t)ns * 32, -1);
  int64_t total = 0;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t width = 0;
    for (int l = 0; l < 32 && s * 32 + l < n; ++l) {
      const int32_t r = order[s * 32 + l];
      S.srow[s * 32 + l] = r;
      width = std::max<int64_t>(width, len(r));
    }
    total += width * 32;
    if (total > INT32_MAX) return false;
    S.sptr[s + 1] = (int32_t)total;
  }
  S.sidx.assign((size_t)total, -1);
  S.src.assign((size_t)total, -1);
  for (int64_t s = 0; s < ns; ++s)
    for (int l = 0; l < 32; ++l) {
      const int32_t r = S.srow[s * 32 + l];
      if (r < 0) continue;
      for (int64_t e = 0; e < len(r); ++e) {
        const int64_t pos = S.sptr[s] + e * 32 + l;
        S.sidx[pos] = M.idx[M.ptr[r] + e];
        S.src[pos] = M.ptr[r] + e;
      }
    }
  return true;
}

static DevCsr upload_csr(std::vector<void*>& owner, const Csr& M, int precisions, const Dia* dia = nullptr,
                         int halo_kb = 0, bool sell = false) {
  DevCsr D;
  if (M.rows > INT32_MAX || M.nnz() > INT32_MAX) fail(AMGSYM_ERR_ARG, "matrix too large for 32-bit device indices");
  D.rows = (int32_t)M.rows;
  D.cols = (int32_t)M.cols;
  D.nnz = M.nnz();
  D.avg_row = M.rows > 0 ? (double)M.nnz() / (double)M.rows : 0.0;
  std::vector<int32_t> p32(M.ptr.begin(), M.ptr.end());
  D.ptr = upload(owner, p32.data(), (int64_t)p32.size());
  D.idx = upload(owner, M.idx.data(), D.nnz);
  if (precisions & 1) D.v64 = upload(owner, M.val.data(), D.nnz);
  if (precisions & 2) {
    std::vector<float> v(M.val.begin(), M.val.end());
    D.v32 = upload(owner, v.data(), D.nnz);
  }
  if (precisions & 4) {
    std::vector<__nv_bfloat16> v(D.nnz);
    for (int64_t i = 0; i < D.nnz; ++i) v[i] = __float2bfloat16((float)M.val[i]);
    D.v16 = upload(owner, v.data(), D.nnz);
  }
  if (dia && dia->ndiag > 0) {
    // the same value conversions as the CSR copies, so both forms multiply
    // by identical numbers
    D.ndiag = dia->ndiag;
    for (int d = 0; d < kMaxDiag; ++d) {
      D.doff[d] = dia->off[d];
      D.dsrc[d] = dia->src[d];
      D.dshift[d] = dia->shift[d];
    }
    // arrays of dstride elements: rows rounded up to 8, zero padded
    const int64_t rows = M.rows;
    D.dstride = (rows + 7) / 8 * 8;
    const int64_t cnt = D.dstride * dia->nstored;
    std::vector<double> padded((size_t)cnt, 0.0);
    for (int q = 0; q < dia->nstored; ++q)
      std::copy(dia->val.begin() + (size_t)q * rows, dia->val.begin() + (size_t)(q + 1) * rows,
                padded.begin() + (size_t)q * D.dstride);
    if (precisions & 1) D.dv64 = upload(owner, padded.data(), cnt);
    if (precisions & 2) {
      std::vector<float> v(padded.begin(), padded.end());
      D.dv32 = upload(owner, v.data(), cnt);
    }
    if (precisions & 4) {
      std::vector<__nv_bfloat16> v(cnt);
      for (int64_t i = 0; i < cnt; ++i) v[i] = __float2bfloat16((float)padded[i]);
      D.dv16 = upload(owner, v.data(), cnt);
    }
  }
  HostHalo H;
  if (D.ndiag == 0 && halo_kb > 0 && build_halo(M, (int64_t)halo_kb * 1024, H)) {
    D.htiles = (int32_t)(H.hptr.size() - 1);
    D.hrows = H.rows;
    D.hmax = H.hmax;
    D.hsum = H.hptr.back();
    D.hptr = upload(owner, H.hptr.data(), (int64_t)H.hptr.size());
    D.hx = upload(owner, H.hx.data(), (int64_t)H.hx.size());
    D.lidx = upload(owner, H.lidx.data(), (int64_t)H.lidx.size());
  }
  HostSell S;
  // rows of a few entries (prolongations: 1-3) ran at half the CSR speed sliced
  if (D.ndiag == 0 && sell && M.nnz() >= 8 * M.rows && build_sell(M, S)) {
    // the same value conversions as the CSR copies (padding: 0)
    D.nslices = (int32_t)(S.sptr.size() - 1);
    D.sentries = (int64_t)S.sidx.size();
    D.sptr = upload(owner, S.sptr.data(), (int64_t)S.sptr.size());
    D.srow = upload(owner, S.srow.data(), (int64_t)S.srow.size());
    D.sidx = upload(owner, S.sidx.data(), D.sentries);
    std::vector<double> v((size_t)D.sentries, 0.0);
    for (int64_t q = 0; q < D.sentries; ++q)
      if (S.src[q] >= 0) v[q] = M.val[S.src[q]];
    if (precisions & 1) D.sv64 = upload(owner, v.data(), D.sentries);
    if (precisions & 2) {
      std::vector<float> f(v.begin(), v.end());
      D.sv32 = upload(owner, f.data(), D.sentries);
    }
    if (precisions & 4) {
      std::vector<__nv_bfloat16> h((size_t)D.sentries);
      for (int64_t q = 0; q < D.sentries; ++q) h[q] = __float2bfloat16((float)v[q]);
      D.sv16 = upload(owner, h.data(), D.sentries);
    }
  }
  return D;
}

static void free_work(Device* D) {
  for (void* p : D->work_owned) cudaFree(p);
  D->work_owned.clear();
  if (D->h_status) cudaFreeHost(D->h_status);
  if (D->h_relres) cudaFreeHost(D->h_relres);
  D->h_status = nullptr;
  D->h_relres = nullptr;
  D->w64 = PrecWork();
  D->w32 = PrecWork();
  D->work_nrhs = 0;
  if (D->graph.exec) cudaGraphExecDestroy(D->graph.exec);
  D->graph = GraphCache();
  D->cycle_plans.clear();  // their phase arrays were work allocations
}

void device_free(amgsym_problem* p) {
  if (p->amgr && p->amgr->coarse) device_free(p->amgr->coarse.get());
  Device* D = p->dev;
  if (!D) return;
  cudaSetDevice(D->device_id);
  cudaDeviceSynchronize();
  free_work(D);
  for (void* q : D->owned) cudaFree(q);
  if (D->cap_stream) cudaStreamDestroy(D->cap_stream);
  for (auto& e : D->ev)
    if (e) cudaEventDestroy(e);
  delete D;
  p->dev = nullptr;
}

// lambda_max(G A G^T) on the device: the steps of the host estimator
// (lambda_max_GAGt: uniform[-1, 1] start from the same seed, 30 power
// iterations, each normalised, the Rayleigh quotient of the last) with FP64
// products on the uploaded matrices.
static double device_lambda_max(Device* D, const DevCsr& A, const DevCsr& G, const DevCsr& Gt, int64_t n,
                                uint64_t seed) {
  std::vector<double> h((size_t)n);
  std::mt19937_64 rng(seed ^ 0x9e3779b97f4a7c15ULL);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (auto& x : h) x = U(rng);
  std::vector<void*> tmp;
  double* v = dalloc<double>(tmp, n);
  double* t1 = dalloc<double>(tmp, n);
  double* t2 = dalloc<double>(tmp, n);
  double* t3 = dalloc<double>(tmp, n);
  double* part = dalloc<double>(tmp, (int64_t)mdot_blocks(n, 1));
  double* s = dalloc<double>(tmp, 1);
  struct Free {
    std::vector<void*>& t;
    ~Free() {
      for (void* q : t) cudaFree(q);
    }
  } fr{tmp};
  CK(cudaMemcpy(v, h.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
  Ctx c{D, 1, VEC_F64, VAL_F64, false, nullptr};
  double lam = 0.0, nv2 = 0.0, num = 0.0;
  for (int it = 0; it < 30; ++it) {
    launch_mdot(v, 0, 1, 1, v, n, 1, part, s, nullptr);
    check_launch();
    CK(cudaMemcpy(&nv2, s, sizeof(double), cudaMemcpyDeviceToHost));
    if (!(nv2 > 0.0)) break;
    const double inv = 1.0 / std::sqrt(nv2);
    CK(cudaMemcpy(s, &inv, sizeof(double), cudaMemcpyHostToDevice));
    launch_colscale(v, s, v, n, 1, nullptr);
    spmm(c, Gt, VAL_F64, VEC_F64, VEC_F64, v, t1, 1.0, 0.0, nullptr, false, nullptr);
    spmm(c, A, VAL_F64, VEC_F64, VEC_F64, t1, t2, 1.0, 0.0, nullptr, false, nullptr);
    spmm(c, G, VAL_F64, VEC_F64, VEC_F64, t2, t3, 1.0, 0.0, nullptr, false, nullptr);
    launch_mdot(v, 0, 1, 1, t3, n, 1, part, s, nullptr);
    check_launch();
    CK(cudaMemcpy(&num, s, sizeof(double), cudaMemcpyDeviceToHost));
    lam = num;
    std::swap(v, t3);
  }
  return lam;
}

void device_upload(amgsym_problem* p) {
  device_free(p);
  auto* D = new Device();
  p->dev = D;
  D->epoch = next_generation();
  CK(cudaGetDevice(&D->device_id));
  D->precisions = p->opts.precisions | 1;  // FP64 operator always (outer residuals)
  D->zmarch = p->opts.zmarch != 0;
  D->nu = p->opts.nu;
  D->singular = p->singular;
  D->s = p->s;
  D->nb = p->nb;
  D->n_b = p->n_b;
  if (p->s > 4) fail(AMGSYM_ERR_ARG, "device path supports s <= 4");
  D->perm = upload(D->owned, p->perm.data(), (int64_t)p->perm.size());
  auto& H = p->H;
  D->lv.resize(H.levels.size());
  for (size_t l = 0; l < H.levels.size(); ++l) {
    HostLevel& L = H.levels[l];
    DevLevel& V = D->lv[l];
    V.n = (int32_t)L.A.rows;
    V.omega = L.omega;
    // level 0 keeps FP64 always (the reduced operator of the outer loop)
    const int hkb = p->opts.halo_kb;
    const bool sl = p->opts.sell != 0;
    V.A = upload_csr(D->owned, L.A, l == 0 ? D->precisions : p->opts.precisions, &L.Adia, hkb, sl);
    if (!L.coarse_inv.empty()) {
      V.cinv = upload(D->owned, L.coarse_inv.data(), (int64_t)L.coarse_inv.size());
    } else {
      V.P = upload_csr(D->owned, L.P, p->opts.precisions, nullptr, hkb, sl);
      V.R = upload_csr(D->owned, L.R, p->opts.precisions, nullptr, hkb, sl);
      V.G = upload_csr(D->owned, L.G, p->opts.precisions, &L.Gdia, hkb, sl);
      V.Gt = upload_csr(D->owned, L.Gt, p->opts.precisions, &L.Gtdia, hkb, sl);
      if (p->opts.lambda_device && !(L.omega > 0.0)) {
        // the damping's lambda_max, deferred by the host setup
        const uint64_t seed = p->opts.seed + 17 * (uint64_t)l;
        if (V.A.v64 && V.G.v64 && V.Gt.v64)
          L.lambda_max = device_lambda_max(D, V.A, V.G, V.Gt, L.A.rows, seed);
        else
          L.lambda_max = lambda_max_GAGt(L.A, L.G, L.Gt, seed);
        L.omega = (L.lambda_max > 0.0) ? p->opts.omega_scale / L.lambda_max : 1.0;
        V.omega = L.omega;
      }
      // a diagonal FSAI factor: the smoother is the diagonal omega g_ii^2
      bool diag = L.G.nnz() == L.G.rows;
      for (int64_t i = 0; diag && i < L.G.rows; ++i) diag = L.G.idx[L.G.ptr[i]] == (int32_t)i;
      if (diag && L.G.rows > 0) {
        std::vector<double> jd((size_t)L.G.rows);
        for (int64_t i = 0; i < L.G.rows; ++i) jd[i] = L.omega * L.G.val[L.G.ptr[i]] * L.G.val[L.G.ptr[i]];
        if (p->opts.precisions & 1) V.jd64 = upload(D->owned, jd.data(), (int64_t)jd.size());
        if (p->opts.precisions & 6) {
          std::vector<float> j32(jd.begin(), jd.end());
          V.jd32 = upload(D->owned, j32.data(), (int64_t)j32.size());
        }
      }
    }
  }
  D->Ainn = D->lv[0].A;
  // interface couplings
  D->iface = upload_iface(D->owned, p->n_b, p->irow, p->icol, p->ivals, p->nb);
  // AMGR top level and its coarse problem
  if (p->amgr) {
    const HostAmgr& M = *p->amgr;
    DevAmgr& G = D->amgr;
    const int hk = p->opts.halo_kb;
    G.Pb = upload_csr(D->owned, M.Pb, D->precisions, nullptr, hk);
    G.Rb = upload_csr(D->owned, M.Rb, D->precisions, nullptr, hk);
    G.GK = upload_csr(D->owned, M.GK, D->precisions, nullptr, hk);
    G.GKt = upload_csr(D->owned, M.GKt, D->precisions, nullptr, hk);
    G.omegaK = M.omegaK;
    G.n_cb = M.n_cb;
    G.jd64 = upload(D->owned, M.jdC.data(), (int64_t)M.jdC.size());
    std::vector<float> j32(M.jdC.begin(), M.jdC.end());
    G.jd32 = upload(D->owned, j32.data(), (int64_t)j32.size());
    amgsym_problem* cp = M.coarse.get();
    cp->opts.precisions = D->precisions;
    device_upload(cp);
    CK(cudaSetDevice(D->device_id));
    G.cd = cp->dev;
    if (p->opts.amgr_sym_ac && p->nb > 1) {
      // the coarse problem's level-0 products in the transformed basis
      auto S = std::make_shared<SymCoarse>();
      S->inn = upload_csr(G.cd->owned, M.Ac0, D->precisions);
      S->iface = upload_iface(G.cd->owned, M.n_cb, M.cirow, M.cicol, M.civals, p->nb);
      S->nb = p->nb;
      S->n_cb = M.n_cb;
      G.cd->symc = S;
    }
    D->has_amgr = true;
  }
  // persistent coarse cycle from the first level below the finest with at
  // most fuse_rows rows (only when it leaves at least one product to fuse)
  D->fuse_level = -1;
  if (p->opts.fuse_rows > 0)
    for (size_t l = 1; l < D->lv.size(); ++l)
      if (D->lv[l].n <= p->opts.fuse_rows) {
        if (!D->lv[l].cinv) D->fuse_level = (int)l;
        break;
      }
  {
    unsigned* words = dalloc<unsigned>(D->owned, 4);
    CK(cudaMemset(words, 0, 4 * sizeof(unsigned)));
    D->bar.count = words;
    D->bar.gen = words + 1;
    D->bar.err = reinterpret_cast<int32_t*>(words + 2);
  }
  CK(cudaStreamCreateWithFlags(&D->cap_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&D->ev[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&D->ev[1], cudaEventDisableTiming));
  CK(cudaDeviceSynchronize());
}

void alloc_scalars(Device* D, DevScalars& sc, int32_t C, int32_t nrhs) {
  sc.rz = dalloc<double>(D->work_owned, C);
  sc.alpha = dalloc<double>(D->work_owned, C);
  sc.beta = dalloc<double>(D->work_owned, C);
  sc.rr = dalloc<double>(D->work_owned, C);
  sc.bnorm2 = dalloc<double>(D->work_owned, nrhs);
  sc.relres = dalloc<double>(D->work_owned, nrhs);
  sc.tol2 = dalloc<double>(D->work_owned, 1);
  sc.active = dalloc<int32_t>(D->work_owned, C);
  sc.status = dalloc<int32_t>(D->work_owned, 4);
  sc.partial_cap = (int64_t)max_grid_blocks() * C;
  sc.partials = dalloc<double>(D->work_owned, sc.partial_cap);
  sc.ticket = dalloc<unsigned>(D->work_owned, 1);
  CK(cudaMemset(sc.ticket, 0, sizeof(unsigned)));
  CK(cudaMemset(sc.status, 0, 4 * sizeof(int32_t)));
}

void ensure_work(Device* D, int32_t nrhs, VecType vt) {
  if (nrhs > D->work_nrhs) {
    CK(cudaDeviceSynchronize());
    free_work(D);
    D->work_gen = next_generation();
    D->work_nrhs = nrhs;
    const int32_t C = nrhs * D->nb;
    D->bh = dalloc<double>(D->work_owned, D->n_b * C);
    D->xh = dalloc<double>(D->work_owned, D->n_b * C);
    alloc_scalars(D, D->sc_out, C, nrhs);
    alloc_scalars(D, D->sc_in, C, nrhs);
    CK(cudaMallocHost(&D->h_status, 8 * sizeof(int32_t)));
    CK(cudaMallocHost(&D->h_relres, sizeof(double) * nrhs));
  }
  PrecWork& W = vt == VEC_F64 ? D->w64 : D->w32;
  if (W.ready) return;
  D->work_gen = next_generation();
  const int32_t C = D->work_nrhs * D->nb;
  const size_t es = vt == VEC_F64 ? 8 : 4;
  auto vec = [&](int64_t rows) -> void* {
    void* p = nullptr;
    if (rows <= 0) return nullptr;
    CK(cudaMalloc(&p, es * (size_t)rows * (size_t)C));
    D->work_owned.push_back(p);
    return p;
  };
  W.lw.resize(D->lv.size());
  for (size_t l = 0; l < D->lv.size(); ++l) {
    const int64_t n = D->lv[l].n;
    if (l > 0) {
      W.lw[l].y = vec(n);
      W.lw[l].z = vec(n);
    }
    W.lw[l].r = vec(n);
    W.lw[l].t = vec(n);
  }
  W.r = vec(D->n_b);
  W.z = vec(D->n_b);
  W.p = vec(D->n_b);
  W.q = vec(D->n_b);
  if (D->symc) {  // [n_cb][nrhs * 2^s]: the same size as the copy layout
    W.sxh = vec(D->n_b);
    W.syh = vec(D->n_b);
  }
  if (D->has_amgr) {
    W.at = vec(D->n_b);
    W.ar = vec(D->n_b);
    W.arc = vec(D->amgr.n_cb);
    W.ahc = vec(D->amgr.n_cb);
    W.arc2 = vec(D->amgr.n_cb);  // n_cb * 2^s rows x nrhs columns: the same size
    W.ahc2 = vec(D->amgr.n_cb);
    ensure_work(D->amgr.cd, D->work_nrhs, vt);
  }
  // FP64 PCG iterates on x^ itself; the FP32 inner PCG on its own correction.
  W.x = vt == VEC_F64 ? (void*)D->xh : vec(D->n_b);
  W.ready = true;
}

// ---------------------------------------------------------------------------
// Kernel sequencing.

// Fixed tile from the row length (what the autotuner picks on the 256^3
// workload, measured on GB300): short rows take one thread per row holding
// two 16-byte vectors of columns (coalesced index/value loads for a warp of
// consecutive rows); medium rows split their entries over 4 lanes; the long
// rows of the coarse Galerkin operators over 4-16 lanes with one vector each.
Tile fixed_tile(const DevCsr& M, int32_t C, VecType xt) {
  const int V = xt == VEC_F64 ? 2 : 4;
  const bool two = C % (2 * V) == 0 && C / (2 * V) >= 1;
  Tile t;
  const double r = M.avg_row;
  if (M.ndiag > 0) {  // diagonal-offset form: one lane per row, two vectors
    t.cpt = two ? 2 * V : V;
    t.kl = 1;
  } else if (r < 10.0) {
    t.cpt = two ? 2 * V : V;
    t.kl = 1;
  } else if (r < 32.0) {
    t.cpt = two ? 2 * V : V;
    t.kl = 4;
  } else if (r < 60.0) {
    t.cpt = V;
    t.kl = 4;
  } else {
    t.cpt = V;
    t.kl = 16;
  }
  if (C % t.cpt) t.cpt = (C % V == 0) ? V : 1;
  const int tpc = C / t.cpt;
  if (tpc & (tpc - 1)) t.kl = 1;
  while (t.kl > 1 && tpc * t.kl > 32) t.kl >>= 1;
  return t;
}


SpmmArgs make_spmm_args(const Ctx& c, const DevCsr& M, ValType mt, VecType xt, VecType ot, const void* X,
                        void* Y, double alpha, double beta, const void* Z, bool iface, const DotArgs* dot) {
  SpmmArgs a;
  a.rows = M.rows;
  a.C = c.C;
  a.ptr = M.ptr;
  a.idx = M.idx;
  a.val = M.vals(mt);
  if (!a.val) fail(AMGSYM_ERR_STATE, "matrix values of the requested precision were not built (opts.precisions)");
  a.X = X;
  a.Y = Y;
  a.Z = Z;
  a.alpha = alpha;
  a.beta = beta;
  if (iface && c.D->iface.mask) {
    a.imask = c.D->iface.mask;
    a.iprefix = c.D->iface.prefix;
    a.iptr = c.D->iface.iptr;
    a.irows = c.D->iface.irows;
    a.nflag = c.D->iface.n_rows_flagged;
    a.icol = c.D->iface.icol;
    const bool f64 = (mt == VAL_F64) || (xt == VEC_F64);
    a.ival = f64 ? (const void*)c.D->iface.ival64 : (const void*)c.D->iface.ival32;
    a.nb = c.D->nb;
  }
  if (M.ndiag > 0 && M.dvals(mt)) {
    a.ndiag = M.ndiag;
    for (int d = 0; d < kMaxDiag; ++d) {
      a.doff[d] = M.doff[d];
      a.dsrc[d] = M.dsrc[d];
      a.dshift[d] = M.dshift[d];
    }
    a.dval = M.dvals(mt);
    a.dstride = M.dstride;
    if (c.D->zmarch) stencil_geometry(M.rows, M.ndiag, M.doff, a);
  }
  if (M.nslices > 0 && a.ndiag == 0 && M.svals(mt)) {
    a.nslices = M.nslices;
    a.sptr = M.sptr;
    a.srow = M.srow;
    a.sidx = M.sidx;
    a.sval = M.svals(mt);
  }
  if (M.htiles > 0 && a.ndiag == 0) {
    a.htiles = M.htiles;
    a.hrows = M.hrows;
    a.hmax = M.hmax;
    a.hptr = M.hptr;
    a.hx = M.hx;
    a.lidx = M.lidx;
  }
  if (dot) a.dot = *dot;
  a.skip = c.skip;
  // the dot-fused variant has its own tile where the tuner timed one
  auto it = c.D->tiles.end();
  if (dot) it = c.D->tiles.find(TileKey{M.idx, c.C, (int)mt, (int)xt, (int)ot, 1});
  if (it == c.D->tiles.end()) it = c.D->tiles.find(TileKey{M.idx, c.C, (int)mt, (int)xt, (int)ot, 0});
  if (it != c.D->tiles.end()) {
    a.kl = it->second.kl;
    a.cpt = it->second.cpt;
  } else {
    const Tile t = fixed_tile(M, c.C, xt);
    a.kl = t.kl;
    a.cpt = t.cpt;
  }
  return a;
}

void spmm(const Ctx& c, const DevCsr& M, ValType mt, VecType xt, VecType ot, const void* X, void* Y, double alpha,
          double beta, const void* Z, bool iface, const DotArgs* dot) {
  const SpmmArgs a = make_spmm_args(c, M, mt, xt, ot, X, Y, alpha, beta, Z, iface, dot);
  run_spmm(c, M, mt, xt, ot, a);
}

// ---------------------------------------------------------------------------
// Tile autotuner.  For every sparse matrix of the V-cycle and the reduced
// operator, at the column count and precisions of the solve, time each
// candidate tile -- columns per thread (one or two 16-byte vectors) times
// entry lanes per row (1..16) -- with CUDA events and keep the fastest.  It
// runs once per (C, precision) before the PCG graph is captured, on scratch
// level vectors (their contents do not matter for timing).  The dot-fused
// products of the PCG iteration (q = A^ p with <p, q>; the last finest-level
// smoother update with <r, z>) are timed as their own variant, since their
// register budget differs from the plain product's.  Results are
// bit-reproducible for a fixed tile choice; the choice itself is timing-based.
void tune_tiles(const Ctx& c) {
  Device* D = c.D;
  auto key = std::make_tuple(c.C, (int)c.vt, (int)c.mt);
  if (D->tuned.count(key)) return;
  PrecWork& W = c.vt == VEC_F64 ? D->w64 : D->w32;
  const size_t es = c.vt == VEC_F64 ? 8 : 4;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (size_t l = 0; l < D->lv.size(); ++l) {
    if (W.lw[l].t) CK(cudaMemsetAsync(W.lw[l].t, 0, es * (size_t)D->lv[l].n * c.C, c.st));
    if (W.lw[l].z) CK(cudaMemsetAsync(W.lw[l].z, 0, es * (size_t)D->lv[l].n * c.C, c.st));
    if (W.lw[l].r) CK(cudaMemsetAsync(W.lw[l].r, 0, es * (size_t)D->lv[l].n * c.C, c.st));
  }
  // dot: the fused-dot variant of the product (with its epilogue operand),
  // timed and stored as its own tile (variant 1): its register budget differs
  struct Job {
    const DevCsr* M;
    ValType mt;
    const void* X;
    void* Y;
    bool iface;
    bool dot = false;
    double beta = 0.0;
    const void* W = nullptr;
  };
  std::vector<Job> jobs;
  const ValType kmt = c.vt == VEC_F64 ? VAL_F64 : VAL_F32;
  jobs.push_back({&D->Ainn, kmt, W.lw[0].t, W.lw[0].r, true});  // reduced operator
  // the PCG's q = A^ p with <p, q>
  jobs.push_back({&D->Ainn, kmt, W.lw[0].t, W.lw[0].r, true, true, 0.0, W.lw[0].t});
  for (size_t l = 0; l + 1 < D->lv.size(); ++l) {
    const DevLevel& L = D->lv[l];
    if (L.cinv) break;
    jobs.push_back({&L.A, c.mt, W.lw[l].t, W.lw[l].r, false});
    jobs.push_back({&L.G, c.mt, W.lw[l].t, W.lw[l].r, false});
    jobs.push_back({&L.Gt, c.mt, W.lw[l].t, W.lw[l].r, false});
    // the last finest-level smoother update z += w G^T (...) with <r, z>: the
    // partner is the PCG's r, as in the solve (level 0 has no level z vector)
    if (l == 0) jobs.push_back({&L.Gt, c.mt, W.lw[l].t, W.lw[l].r, false, true, 1.0, W.r});
    jobs.push_back({&L.R, c.mt, W.lw[l].r, W.lw[l + 1].y, false});
    jobs.push_back({&L.P, c.mt, W.lw[l + 1].z, W.lw[l].t, false});
  }
  const int vmax = c.vt == VEC_F64 ? 2 : 4;
  for (const Job& j : jobs) {
    if (!j.M->vals(j.mt)) continue;
    if (!j.X || !j.Y || (j.dot && !j.W))
      fail(AMGSYM_ERR_STATE, "tile tuner: a work vector of a timed product is missing");
    Tile best;
    float best_ms = 1e30f;
    for (int cm = 1; cm <= 2; ++cm) {
      const int cpt = vmax * cm;
      if (c.C % cpt) continue;
      const int tpc = c.C / cpt;
      for (int kl = 1; kl <= 16; kl *= 2) {
        if (kl > 1 && ((tpc & (tpc - 1)) || tpc * kl > 32 || j.M->ndiag > 0)) break;
        Ctx cc = c;
        const int var = j.dot ? 1 : 0;
        D->tiles[TileKey{j.M->idx, c.C, (int)j.mt, (int)c.vt, (int)c.vt, var}] = Tile{cpt, kl};
        DotArgs dj;  // per-column sums only (no finalisation), on the solve's scratch partials
        dj.mode = DOT_WY;
        dj.final = FIN_NONE;
        dj.W = j.W;
        dj.sc = D->sc_out;
        const DotArgs* dp = j.dot ? &dj : nullptr;
        const void* Zj = j.beta != 0.0 ? j.Y : nullptr;
        spmm(cc, *j.M, j.mt, c.vt, c.vt, j.X, j.Y, 1.0, j.beta, Zj, j.iface, dp);  // warm-up
        CK(cudaEventRecord(e0, c.st));
        const int reps = 3;
        for (int r = 0; r < reps; ++r) spmm(cc, *j.M, j.mt, c.vt, c.vt, j.X, j.Y, 1.0, j.beta, Zj, j.iface, dp);
        CK(cudaEventRecord(e1, c.st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms * 0.97f) {  // prefer the earlier (simpler) tile on near-ties
          best_ms = ms;
          best = Tile{cpt, kl};
        }
      }
    }
    if (best.cpt > 0) {
      // the same tile serves every output type of this matrix and variant
      const int var = j.dot ? 1 : 0;
      D->tiles[TileKey{j.M->idx, c.C, (int)j.mt, (int)c.vt, (int)c.vt, var}] = best;
      D->tiles[TileKey{j.M->idx, c.C, (int)j.mt, (int)c.vt, (int)VEC_F32, var}] = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  D->tuned.insert(key);
  D->tiles_gen++;
}

// ---------------------------------------------------------------------------
// Smoother steps of the V-cycle (presmoothing from zero, then sweeps), with
// the FSAI factor G_l of the level: z = w G^T G y and z += w G^T G (y - A z).
// A diagonal G (one entry per row) is applied as the diagonal jd = w g_ii^2
// in one elementwise kernel instead of two products.  `dot` (the fused
// <r, z> of the final level-0 product) keeps the product form.

static int level_of(const Ctx& c, const DevLevel& L) { return (int)(&L - c.D->lv.data()); }

static void run_jacobi(const Ctx& c, const DevLevel& L, const void* jd, const void* src, void* z, int accumulate) {
  ProfScope ps(c.st);
  launch_jacobi(c.vt, L.n, c.C, jd, src, z, accumulate, c.st, c.skip);
  check_launch();
  if (ps.on())
    ps.end(std::string("jacobi_kernel<") + tname(c.vt) + ">",
           "L" + std::to_string(level_of(c, L)) + (accumulate ? " diagonal smoother z += D r" : " diagonal smoother z = D y"),
           level_of(c, L), xsize(c.vt) * (int64_t)L.n * (1 + (int64_t)c.C * (accumulate ? 3 : 2)));
}

// r = y - A_l z.  On level 0 of the AMGR coarse problem with its
// transformed-basis operator (SymCoarse): butterfly z to the transformed
// layout, the reduced SpMM with the coarse couplings, and the scaled
// butterfly back with the residual epilogue.
static void level_residual(const Ctx& c, const DevLevel& L, const void* z, void* r, const void* y, bool hat) {
  Device* D = c.D;
  if (D->symc && &L == &D->lv[0]) {
    const SymCoarse& S = *D->symc;
    PrecWork& W = c.vt == VEC_F64 ? D->w64 : D->w32;
    const int32_t nrhs = c.C;  // the coarse problem has one column per right-hand side
    {
      ProfScope ps(c.st);
      launch_coarse_relayout(c.vt, z, W.sxh, S.n_cb, nrhs, S.nb, 1, c.st);
      check_launch();
      if (ps.on())
        ps.end(std::string("coarse_relayout_kernel<") + tname(c.vt) + ">", "AMGR A_c: to the transformed basis", 0,
               2 * xsize(c.vt) * S.n_cb * S.nb * nrhs);
    }
    Ctx ch = c;
    ch.C = nrhs * S.nb;
    SpmmArgs a = make_spmm_args(ch, S.inn, c.mt, c.vt, c.vt, W.sxh, W.syh, 1.0, 0.0, nullptr, false, nullptr);
    if (S.iface.mask) {
      a.imask = S.iface.mask;
      a.iprefix = S.iface.prefix;
      a.iptr = S.iface.iptr;
      a.irows = S.iface.irows;
      a.nflag = S.iface.n_rows_flagged;
      a.icol = S.iface.icol;
      a.ival = (c.mt == VAL_F64 || c.vt == VEC_F64) ? (const void*)S.iface.ival64 : (const void*)S.iface.ival32;
      a.nb = S.nb;
    }
    run_spmm(ch, S.inn, c.mt, c.vt, c.vt, a);
    {
      ProfScope ps(c.st);
      launch_coarse_relayout(c.vt, W.syh, r, S.n_cb, nrhs, S.nb, 0, c.st, -1.0, 1.0, y);
      check_launch();
      if (ps.on())
        ps.end(std::string("coarse_relayout_kernel<") + tname(c.vt) + ">", "AMGR A_c: back, r = y - A_c z", 0,
               3 * xsize(c.vt) * S.n_cb * S.nb * nrhs);
    }
    return;
  }
  spmm(c, L.A, c.mt, c.vt, c.vt, z, r, -1.0, 1.0, y, hat, nullptr);
}

static void smooth_first(const Ctx& c, const DevLevel& L, LevelWork& lw, const void* y, void* z) {
  if (const void* jd = L.jd(c.vt)) {
    run_jacobi(c, L, jd, y, z, 0);
    return;
  }
  spmm(c, L.G, c.mt, c.vt, c.vt, y, lw.t, 1.0, 0.0, nullptr, false, nullptr);
  spmm(c, L.Gt, c.mt, c.vt, c.vt, lw.t, z, L.omega, 0.0, nullptr, false, nullptr);
}

static void smooth_sweep(const Ctx& c, const DevLevel& L, LevelWork& lw, const void* y, void* z, bool hat,
                         const DotArgs* dot) {
  level_residual(c, L, z, lw.r, y, hat);
  const void* jd = L.jd(c.vt);
  if (jd && !dot) {
    run_jacobi(c, L, jd, lw.r, z, 1);
    return;
  }
  spmm(c, L.G, c.mt, c.vt, c.vt, lw.r, lw.t, 1.0, 0.0, nullptr, false, nullptr);
  spmm(c, L.Gt, c.mt, c.vt, c.vt, lw.t, z, L.omega, 1.0, z, false, dot);
}

// ---------------------------------------------------------------------------
// Persistent coarse cycle (k_cycle.cu).  The phases are the products of
// vcycle() below from level Device::fuse_level down, in the same order with
// the same arguments, entry lanes and therefore the same sums.

static void cycle_phase(const Ctx& c, std::vector<CyclePhase>& out, const DevCsr& M, const void* X, void* Y,
                        double alpha, double beta, const void* Z, int kcpt) {
  CyclePhase ph;
  ph.kind = CYCLE_SPMM;
  ph.a = make_spmm_args(c, M, c.mt, c.vt, c.vt, X, Y, alpha, beta, Z, false, nullptr);
  ph.a.skip = nullptr;
  int cpt = 0, kl = 1;
  spmm_resolved_tile(c.vt, c.vt, ph.a, &cpt, &kl);
  // the kernel's own column split; entry lanes as the stand-alone launch
  const int tpc = c.C / kcpt;
  if (tpc & (tpc - 1)) kl = 1;
  while (kl > 1 && tpc * kl > 32) kl >>= 1;
  ph.a.kl = kl;
  ph.a.cpt = kcpt;
  out.push_back(ph);
}

static void cycle_phases(const Ctx& c, int l, const void* y, void* z, int kcpt, std::vector<CyclePhase>& out) {
  Device* D = c.D;
  const DevLevel& L = D->lv[l];
  PrecWork& W = c.vt == VEC_F64 ? D->w64 : D->w32;
  LevelWork& lw = W.lw[l];
  if (L.cinv) {
    CyclePhase ph;
    ph.kind = CYCLE_DENSE;
    ph.c.n = L.n;
    ph.c.C = c.C;
    ph.c.Ainv = L.cinv;
    ph.c.Y = y;
    ph.c.Z = z;
    out.push_back(ph);
    return;
  }
  // the smoother steps of smooth_first / smooth_sweep
  const void* jd = L.jd(c.vt);
  auto jacobi = [&](const void* src, int accumulate) {
    CyclePhase ph;
    ph.kind = CYCLE_JACOBI;
    ph.j.rows = L.n;
    ph.j.C = c.C;
    ph.j.accumulate = accumulate;
    ph.j.jd = jd;
    ph.j.src = src;
    ph.j.z = z;
    out.push_back(ph);
  };
  auto sweep = [&]() {
    cycle_phase(c, out, L.A, z, lw.r, -1.0, 1.0, y, kcpt);
    if (jd) {
      jacobi(lw.r, 1);
    } else {
      cycle_phase(c, out, L.G, lw.r, lw.t, 1.0, 0.0, nullptr, kcpt);
      cycle_phase(c, out, L.Gt, lw.t, z, L.omega, 1.0, z, kcpt);
    }
  };
  if (jd) {
    jacobi(y, 0);
  } else {
    cycle_phase(c, out, L.G, y, lw.t, 1.0, 0.0, nullptr, kcpt);
    cycle_phase(c, out, L.Gt, lw.t, z, L.omega, 0.0, nullptr, kcpt);
  }
  for (int k = 1; k < D->nu; ++k) sweep();
  cycle_phase(c, out, L.A, z, lw.r, -1.0, 1.0, y, kcpt);
  LevelWork& cw = W.lw[l + 1];
  cycle_phase(c, out, L.R, lw.r, cw.y, 1.0, 0.0, nullptr, kcpt);
  cycle_phases(c, l + 1, cw.y, cw.z, kcpt, out);
  cycle_phase(c, out, L.P, cw.z, z, 1.0, 1.0, z, kcpt);
  for (int k = 0; k < D->nu; ++k) sweep();
}

static CycleKey cycle_key(const Ctx& c) {
  return CycleKey{c.C, (int)c.vt, (int)c.mt, c.D->work_gen, c.D->tiles_gen};
}

// Whether a cooperative launch works here and can be captured in a graph:
// one capture of an empty launch (no phases: the kernel returns at once).
static bool coop_supported(Device* D, const Ctx& c) {
  if (D->coop_ok >= 0) return D->coop_ok == 1;
  D->coop_ok = 0;
  const int grid = cycle_grid(c.mt, c.vt, c.C);
  if (grid < 1) return false;
  int attr = 0;
  if (cudaDeviceGetAttribute(&attr, cudaDevAttrCooperativeLaunch, D->device_id) != cudaSuccess || !attr) {
    (void)cudaGetLastError();
    return false;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  bool ok = cudaStreamBeginCapture(D->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const cudaError_t le = launch_cycle(c.mt, c.vt, c.C, grid, nullptr, 0, D->bar, nullptr, D->cap_stream);
    count_launch(-1);
    const cudaError_t ee = cudaStreamEndCapture(D->cap_stream, &g);
    ok = le == cudaSuccess && ee == cudaSuccess && g != nullptr;
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  }
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  (void)cudaGetLastError();
  D->coop_ok = ok ? 1 : 0;
  return ok;
}

void prepare_cycle(const Ctx& c) {
  Device* D = c.D;
  if (!c.fuse || D->fuse_level < 1) return;
  const CycleKey key = cycle_key(c);
  if (D->cycle_plans.count(key)) return;
  if (!coop_supported(D, c)) return;
  std::vector<CyclePhase> ph;
  PrecWork& W = c.vt == VEC_F64 ? D->w64 : D->w32;
  const int l = D->fuse_level;
  cycle_phases(c, l, W.lw[l].y, W.lw[l].z, cycle_cpt(c.vt, c.C), ph);
  CyclePlan plan;
  plan.grid = cycle_grid(c.mt, c.vt, c.C);
  plan.nphases = (int32_t)ph.size();
  plan.phases = dalloc<CyclePhase>(D->work_owned, plan.nphases);
  CK(cudaMemcpy(plan.phases, ph.data(), sizeof(CyclePhase) * ph.size(), cudaMemcpyHostToDevice));
  D->cycle_plans[key] = plan;
}

void check_cycle_error(Device* D, cudaStream_t st) {
  if (D->fuse_level < 1 || D->cycle_plans.empty()) return;
  int32_t err = 0;
  CK(cudaMemcpyAsync(&err, D->bar.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) {
    CK(cudaMemset(D->bar.count, 0, 4 * sizeof(unsigned)));
    fail(AMGSYM_ERR_DEVICE_TIMEOUT, "coarse-cycle kernel: a grid-barrier wait ran out (the launch stopped early)");
  }
}

// One V(nu, nu) cycle at level l: z = M_l^{-1} y (Alg. "apply" shape with the
// A_inn hierarchy; presmoothing from zero).  `last` is the optional fused dot
// of the final level-0 kernel.
// The body of one V-cycle level, shared by vcycle() and the no-alloc
// V-cycle (`lws`: the level work vectors; `sub`: the next level's cycle,
// returning where it left z_{l+1}).  Returns the vector holding z on exit.
// pre_done: z already holds the presmoothing from zero (written by the
// restriction of the level above).  On a level whose G is diagonal the next
// level's presmoothing is fused into this level's restriction, and (below
// the finest level) the last postsmoothing into its residual, which then
// writes the new z into lw.t: the diagonal steps cost no launch of their own.
template <typename Sub>
static const void* vcycle_level(const Ctx& c, std::vector<LevelWork>& lws, int l, const void* y, void* z,
                                const DotArgs* last, bool pre_done, Sub&& sub) {
  Device* D = c.D;
  const DevLevel& L = D->lv[l];
  LevelWork& lw = lws[l];
  if (L.cinv) {
    {
      ProfScope ps(c.st);
      launch_coarse_solve(c.vt, L.n, c.C, L.cinv, y, z, c.st, c.skip);
      check_launch();
      if (ps.on())
        ps.end(std::string("coarse_kernel<") + tname(c.vt) + ">", "L" + std::to_string(l) + " dense coarsest solve",
               l, 8 * (int64_t)L.n * L.n + 2 * xsize(c.vt) * (int64_t)L.n * c.C);
    }
    if (last) {
      ProfScope ps(c.st);
      launch_dot(c.vt, L.n, c.C, last->W, z, *last, c.st, c.skip);
      check_launch();
      if (ps.on())
        ps.end(std::string("dot_kernel<") + tname(c.vt) + ">", "L" + std::to_string(l) + " <w,z>", l,
               2 * xsize(c.vt) * (int64_t)L.n * c.C);
    }
    return z;
  }
  const bool hat = c.finest_hat && l == 0;
  const ValType mt = c.mt;
  const VecType vt = c.vt;
  // presmoothing: the first sweep from zero is z = w G^T G y
  if (!pre_done) smooth_first(c, L, lw, y, z);
  for (int k = 1; k < D->nu; ++k) smooth_sweep(c, L, lw, y, z, hat, nullptr);
  // residual and restriction r_c = P^T (y - A z)
  level_residual(c, L, z, lw.r, y, hat);
  LevelWork& cw = lws[l + 1];
  const DevLevel& Lc = D->lv[l + 1];
  const bool persist_next = c.fuse && l + 1 == D->fuse_level;
  const bool fuse_pre = Lc.jd(vt) && !Lc.cinv && !persist_next;
  {
    SpmmArgs a = make_spmm_args(c, L.R, mt, vt, vt, lw.r, cw.y, 1.0, 0.0, nullptr, false, nullptr);
    if (fuse_pre) {
      a.jmode = 1;
      a.jd = Lc.jd(vt);
      a.Y2 = cw.z;
    }
    run_spmm(c, L.R, mt, vt, vt, a);
  }
  const void* zc = sub(l + 1, cw.y, cw.z, fuse_pre);
  // prolongation and update z += P z_c
  spmm(c, L.P, mt, vt, vt, zc, z, 1.0, 1.0, z, false, nullptr);
  // postsmoothing
  const void* jd = L.jd(vt);
  const bool fuse_post = jd && l > 0 && !(last && D->nu >= 1);
  for (int k = 0; k < D->nu; ++k) {
    const bool fin = k == D->nu - 1;
    if (fin && fuse_post) {
      SpmmArgs a = make_spmm_args(c, L.A, mt, vt, vt, z, lw.t, -1.0, 1.0, y, hat, nullptr);
      a.jmode = 2;
      a.jd = jd;
      run_spmm(c, L.A, mt, vt, vt, a);
      return lw.t;
    }
    smooth_sweep(c, L, lw, y, z, hat, fin ? last : nullptr);
  }
  return z;
}

// One V(nu, nu) cycle at level l: z = M_l^{-1} y (Alg. "apply" shape with the
// A_inn hierarchy; presmoothing from zero).  `last` is the optional fused dot
// of the final level-0 kernel.  Returns the vector that holds z_l on exit
// (z, or the level's t after a fused diagonal postsmoothing, never at l = 0).
static const void* vcycle(const Ctx& c, int l, const void* y, void* z, const DotArgs* last, bool pre_done = false) {
  Device* D = c.D;
  PrecWork& W = c.vt == VEC_F64 ? D->w64 : D->w32;
  if (c.fuse && l == D->fuse_level && !last) {
    auto it = D->cycle_plans.find(cycle_key(c));
    if (it != D->cycle_plans.end()) {
      const CyclePlan& pl = it->second;
      const cudaError_t e = launch_cycle(c.mt, c.vt, c.C, pl.grid, pl.phases, pl.nphases, D->bar, c.skip, c.st);
      if (e != cudaSuccess) fail(AMGSYM_ERR_CUDA, std::string("coarse-cycle launch: ") + cudaGetErrorString(e));
      return z;
    }
  }
  return vcycle_level(c, W.lw, l, y, z, last, pre_done, [&](int l1, const void* y1, void* z1, bool pd) {
    return vcycle(c, l1, y1, z1, nullptr, pd);
  });
}

void vcycle_apply(const Ctx& c, const void* R, void* Z) {
  prepare_cycle(c);
  vcycle(c, 0, R, Z, nullptr);
}

// AMGR V(1,1) of Alg. "apply" in the transformed basis: every operator of
// its first level is the same for all 2^s blocks (P = I (x) P_b, the block
// FSAI smoother of eq. "topsmoother"), the residuals use A^_i, and the coarse
// correction solves A_c over the full coarse domain with its AMG hierarchy.
void amgr_apply(const Ctx& c, const void* y, void* z) {
  Device* D = c.D;
  const DevAmgr& M = D->amgr;
  PrecWork& W = c.vt == VEC_F64 ? D->w64 : D->w32;
  const ValType mt = c.mt;
  const VecType vt = c.vt;
  const int32_t nrhs = c.C / D->nb;
  auto smooth = [&](const void* src, double beta) {  // z = beta z + S src
    spmm(c, M.GK, mt, vt, vt, src, W.at, 1.0, 0.0, nullptr, false, nullptr);
    spmm(c, M.GKt, mt, vt, vt, W.at, z, M.omegaK, beta, z, false, nullptr);
    ProfScope ps(c.st);
    launch_jacobi(vt, D->n_b, c.C, M.jd(vt), src, z, 1, c.st, c.skip);
    check_launch();
    if (ps.on())
      ps.end(std::string("jacobi_kernel<") + tname(vt) + ">", "AMGR coarse-point smoother", 0,
             xsize(vt) * D->n_b * (1 + 3 * (int64_t)c.C));
  };
  smooth(y, 0.0);  // presmoothing from zero
  spmm(c, D->Ainn, mt, vt, vt, z, W.ar, -1.0, 1.0, y, true, nullptr);  // r = y - A^ z
  spmm(c, M.Rb, mt, vt, vt, W.ar, W.arc, 1.0, 0.0, nullptr, false, nullptr);
  launch_coarse_relayout(vt, W.arc, W.arc2, M.n_cb, nrhs, D->nb, 0, c.st);
  check_launch();
  Ctx cc{M.cd, nrhs, vt, mt, false, c.st};
  cc.skip = c.skip;
  const void* hc2 = vcycle(cc, 0, W.arc2, W.ahc2, nullptr);
  launch_coarse_relayout(vt, hc2, W.ahc, M.n_cb, nrhs, D->nb, 1, c.st);
  check_launch();
  spmm(c, M.Pb, mt, vt, vt, W.ahc, z, 1.0, 1.0, z, false, nullptr);  // z += P h_c
  spmm(c, D->Ainn, mt, vt, vt, z, W.ar, -1.0, 1.0, y, true, nullptr);
  smooth(W.ar, 1.0);  // postsmoothing
}

// The preconditioner step of the PCG: z = M r with <r, z> (dot `d`).  AMGR
// is not block diagonal in the transformed basis (the AMG of A_c over the
// full coarse domain does not keep the mirror symmetry), so with it the PCG
// is one CG per RHS over all its blocks (DotArgs::coupled).
static void precondition(const Ctx& c, const void* r, void* z, const DotArgs* d) {
  if (c.pc == AMGSYM_PC_AMGR) {
    amgr_apply(c, r, z);
    ProfScope ps(c.st);
    launch_dot(c.vt, c.D->n_b, c.C, r, z, *d, c.st, c.skip);
    check_launch();
    if (ps.on()) ps.end(std::string("dot_kernel<") + tname(c.vt) + ">", "<r,z>", -1, 2 * xsize(c.vt) * c.D->n_b * c.C);
    return;
  }
  vcycle(c, 0, r, z, d);
}

DotArgs make_dot(const DevScalars& sc, int mode, int final, const void* W, int32_t nrhs, int32_t nb,
                        double /*tol: the device scalar sc.tol2 holds it*/, int count_iter) {
  DotArgs d;
  d.mode = mode;
  d.final = final;
  d.W = W;
  d.sc = sc;
  d.cp.nrhs = nrhs;
  d.cp.nb = nb;
  d.cp.count_iter = count_iter;
  return d;
}

// One PCG iteration on vectors of W (precision c.vt):
// q = A^ p (alpha), x += alpha p, r -= alpha q (convergence), z = M r (beta), p = z + beta p.
static void pcg_iteration(const Ctx& c, PrecWork& W, const DevScalars& sc, int32_t nrhs, double tol) {
  Device* D = c.D;
  const ValType kmt = c.vt == VEC_F64 ? VAL_F64 : VAL_F32;  // reduced operator precision
  DotArgs dpq = make_dot(sc, DOT_WY, FIN_ALPHA, W.p, nrhs, D->nb, tol, 0);
  dpq.coupled = c.pc == AMGSYM_PC_AMGR;
  spmm(c, D->Ainn, kmt, c.vt, c.vt, W.p, W.q, 1.0, 0.0, nullptr, true, &dpq);
  DotArgs drr = make_dot(sc, DOT_YY, FIN_CONV, nullptr, nrhs, D->nb, tol, 1);
  {
    ProfScope ps(c.st);
    launch_cg_update1(c.vt, D->n_b, c.C, W.x, W.r, W.p, W.q, drr, c.st, c.skip);
    check_launch();
    if (ps.on())
      ps.end(std::string("cg_update1_kernel<") + tname(c.vt) + ">", "x += a p, r -= a q, <r,r>", -1,
             6 * xsize(c.vt) * D->n_b * c.C);
  }
  DotArgs drz = make_dot(sc, DOT_WY, FIN_BETA, W.r, nrhs, D->nb, tol, 0);
  drz.coupled = c.pc == AMGSYM_PC_AMGR;
  precondition(c, W.r, W.z, &drz);
  {
    ProfScope ps(c.st);
    launch_cg_update2(c.vt, D->n_b, c.C, W.p, W.z, sc.beta, c.st, c.skip);
    check_launch();
    if (ps.on())
      ps.end(std::string("cg_update2_kernel<") + tname(c.vt) + ">", "p = z + b p", -1, 3 * xsize(c.vt) * D->n_b * c.C);
  }
}

void read_status(Device* D, const DevScalars& sc, cudaStream_t st, int32_t* out4) {
  CK(cudaMemcpyAsync(D->h_status, sc.status, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::memcpy(out4, D->h_status, 4 * sizeof(int32_t));
}

// PCG loop until every RHS of `sc` is inactive or maxit; returns iterations.
// The host runs one iteration ahead: it enqueues iteration k + 1 before
// waiting for the status of iteration k.  Kernels of an iteration that starts
// after convergence exit at once (Ctx::skip), so the look-ahead costs only
// launch latency and the GPU never idles on the host's check.
static int pcg_loop(const Ctx& c0, PrecWork& W, const DevScalars& sc, int32_t nrhs, double tol, int maxit,
                    bool use_graph, int graph_mode, bool* breakdown) {
  Device* D = c0.D;
  if (c0.tune) tune_tiles(c0);
  prepare_cycle(c0);
  Ctx c = c0;
  c.skip = sc.status;
  GraphKey graph_key;
  graph_key.mode = graph_mode;
  graph_key.nrhs = nrhs;
  graph_key.tiles_gen = D->tiles_gen;
  // start: z = M r, rz, p = z
  DotArgs drz = make_dot(sc, DOT_WY, FIN_STORE_RZ, W.r, nrhs, D->nb, tol, 0);
  drz.coupled = c.pc == AMGSYM_PC_AMGR;
  precondition(c, W.r, W.z, &drz);
  launch_copy(c.vt, D->n_b * c.C, W.p, W.z, c.st);
  check_launch();
  cudaGraphExec_t exec = nullptr;
  if (use_graph) {
    if (D->graph.exec && D->graph.key == graph_key) {
      exec = D->graph.exec;
    } else {
      if (D->graph.exec) cudaGraphExecDestroy(D->graph.exec);
      D->graph = GraphCache();
      Ctx cc = c;
      cc.st = D->cap_stream;
      cudaGraph_t g = nullptr;
      const int64_t before = launch_count();
      CK(cudaStreamBeginCapture(D->cap_stream, cudaStreamCaptureModeThreadLocal));
      try {
        pcg_iteration(cc, W, sc, nrhs, tol);
      } catch (...) {
        cudaStreamEndCapture(D->cap_stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      CK(cudaStreamEndCapture(D->cap_stream, &g));
      D->graph_kernels = launch_count() - before;
      count_launch(-D->graph_kernels);  // captured, not executed
      CK(cudaGraphInstantiate(&exec, g, 0));
      cudaGraphDestroy(g);
      D->graph.exec = exec;
      D->graph.key = graph_key;
    }
  }
  *breakdown = false;
  int done_at = -1;
  auto check = [&](int k) -> bool {  // status after iteration k (0-based)
    CK(cudaEventSynchronize(D->ev[k & 1]));
    const int32_t* st4 = D->h_status + 4 * (k & 1);
    if (st4[1]) *breakdown = true;
    if (st4[1] || st4[0] == 0) {
      done_at = k + 1;
      return true;
    }
    return false;
  };
  int it = 0;
  for (it = 0; it < maxit; ++it) {
    if (exec) {
      CK(cudaGraphLaunch(exec, c.st));
      count_launch(D->graph_kernels);
    } else {
      pcg_iteration(c, W, sc, nrhs, tol);
    }
    CK(cudaMemcpyAsync(D->h_status + 4 * (it & 1), sc.status, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    CK(cudaEventRecord(D->ev[it & 1], c.st));
    if (it >= 1 && check(it - 1)) break;
  }
  if (done_at < 0 && it > 0) {
    // maxit reached: the last iteration's status decides
    if (!check(it - 1)) done_at = maxit;
  }
  CK(cudaStreamSynchronize(c.st));
  check_cycle_error(D, c.st);
  return done_at < 0 ? maxit : done_at;
}

void check_ptr(const void* p, const char* what) {
  if (!p) fail(AMGSYM_ERR_ARG, std::string(what) + " is NULL");
  if (((uintptr_t)p) % 16) fail(AMGSYM_ERR_ARG, std::string(what) + " must be 16-byte aligned");
}

Device* require_dev(amgsym_t h) {
  if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
  if (!h->dev) fail(AMGSYM_ERR_STATE, "problem is not on the device (call amgsym_setup without host_only)");
  CK(cudaSetDevice(h->dev->device_id));
  return h->dev;
}

static amgsym_status solve_impl(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                const amgsym_solve_opts* sopts, void* stream, amgsym_solve_info* info) {
  Device* D = require_dev(h);
  amgsym_solve_opts o;
  amgsym_solve_opts_default(&o);
  if (sopts) o = *sopts;
  if (nrhs < 1) fail(AMGSYM_ERR_ARG, "nrhs must be >= 1");
  if (ld < h->n) fail(AMGSYM_ERR_ARG, "ld must be >= n");
  if (!b_dev || !x_dev) fail(AMGSYM_ERR_ARG, "NULL vector");
  if ((int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be <= 256 per call");
  if (!(o.tol > 0.0)) fail(AMGSYM_ERR_ARG, "tol must be positive");
  if (o.maxit < 1) fail(AMGSYM_ERR_ARG, "maxit must be >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool mixed = o.precision != AMGSYM_PREC_FP64;
  const VecType vt = mixed ? VEC_F32 : VEC_F64;
  const ValType vmt = o.precision == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : mixed ? VAL_F32 : VAL_F64;
  if (mixed && !(h->opts.precisions & (o.precision == AMGSYM_PREC_MIXED_BF16 ? 4 : 2)))
    fail(AMGSYM_ERR_STATE, "setup did not build the value precision this mode needs (opts.precisions)");
  if (o.preconditioner != AMGSYM_PC_AMG && o.preconditioner != AMGSYM_PC_AMGR)
    fail(AMGSYM_ERR_ARG, "unknown preconditioner");
  if (o.preconditioner == AMGSYM_PC_AMGR && !D->has_amgr)
    fail(AMGSYM_ERR_STATE, "AMGR was not built: call amgsym_setup with opts.amgr = 1");
  ensure_work(D, nrhs, vt);
  const int32_t C = nrhs * D->nb;
  Ctx c{D, C, vt, vmt, o.finest_hat != 0, st};
  c.tune = o.tune != 0;
  c.fuse = true;
  c.pc = o.preconditioner;
  Ctx c64{D, C, VEC_F64, VAL_F64, false, st};
  // 64-bit work is needed for the FP64 path; the mixed path uses bh/xh only.
  PrecWork& W = mixed ? D->w32 : D->w64;
  // Forward transform and reference norms.
  launch_transform_fwd(b_dev, nrhs, ld, D->perm, D->n_b, D->s, D->bh, VEC_F64, st);
  check_launch();
  if (D->singular) {
    // the compatible part of b: its constant component removed
    launch_sub_block0_mean(D->bh, D->n_b, nrhs, D->nb, D->sc_out.partials, D->sc_out.partial_cap, st);
    check_launch();
  }
  DotArgs dbn = make_dot(D->sc_out, DOT_WY, FIN_STORE_BN, nullptr, nrhs, D->nb, o.tol, 0);
  launch_dot(VEC_F64, D->n_b, C, D->bh, D->bh, dbn, st);
  check_launch();
  launch_init_scalars(D->sc_out, nrhs, D->nb, st);
  check_launch();
  launch_set_value(D->sc_out.tol2, o.tol * o.tol, st);
  check_launch();
  if (o.use_x0) {
    launch_transform_fwd(x_dev, nrhs, ld, D->perm, D->n_b, D->s, D->xh, VEC_F64, st);
  } else {
    launch_zero(VEC_F64, D->n_b * C, D->xh, st);
  }
  check_launch();
  const bool graphs = o.use_graph != 0;
  int total_it = 0, outer = 0;
  bool breakdown = false;
  int32_t st4[4];
  amgsym_status result = AMGSYM_OK;
  if (!mixed) {
    // FP64 PCG with up to two restarts from the true residual (reading of
    // the stopping rule: recurrence residual, confirmed by b^ - A^ x^).
    for (int restart = 0; restart < 3; ++restart) {
      launch_init_scalars(D->sc_out, nrhs, D->nb, st);
      DotArgs drr = make_dot(D->sc_out, DOT_YY, FIN_CONV, nullptr, nrhs, D->nb, o.tol, 0);
      spmm(c64, D->Ainn, VAL_F64, VEC_F64, VEC_F64, D->xh, W.r, -1.0, 1.0, D->bh, true, &drr);
      read_status(D, D->sc_out, st, st4);
      if (st4[0] == 0 || total_it >= o.maxit) break;
      const int it = pcg_loop(c, W, D->sc_out, nrhs, o.tol, o.maxit - total_it, graphs,
                              0x100 | (o.finest_hat ? 1 : 0) | (o.preconditioner << 4), &breakdown);
      total_it += it;
      if (breakdown) break;
    }
    if (!breakdown) {
      // final true residual
      launch_init_scalars(D->sc_out, nrhs, D->nb, st);
      DotArgs drr = make_dot(D->sc_out, DOT_YY, FIN_CONV, nullptr, nrhs, D->nb, o.tol, 0);
      spmm(c64, D->Ainn, VAL_F64, VEC_F64, VEC_F64, D->xh, W.r, -1.0, 1.0, D->bh, true, &drr);
      read_status(D, D->sc_out, st, st4);
    }
  } else {
    // FP64 iterative refinement around the FP32 inner PCG.
    for (outer = 0; outer <= o.max_outer; ++outer) {
      DotArgs drr = make_dot(D->sc_out, DOT_YY, FIN_CONV, nullptr, nrhs, D->nb, o.tol, 0);
      // r32 = float(b^ - A^ x^), FP64 arithmetic
      spmm(c64, D->Ainn, VAL_F64, VEC_F64, VEC_F32, D->xh, W.r, -1.0, 1.0, D->bh, true, &drr);
      read_status(D, D->sc_out, st, st4);
      if (st4[0] == 0 || outer == o.max_outer || total_it >= o.maxit) break;
      // Inner target: only as much reduction as the remaining distance to tol
      // needs (with a 4x margin), but at least inner_tol, at most 0.5.
      CK(cudaMemcpyAsync(D->h_relres, D->sc_out.relres, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      double worst = 0.0;
      for (int r = 0; r < nrhs; ++r) worst = std::max(worst, D->h_relres[r]);
      double eta = worst > 0.0 ? 0.25 * o.tol / worst : o.inner_tol;
      eta = std::min(0.5, std::max(o.inner_tol, eta));
      launch_set_value(D->sc_in.tol2, eta * eta, st);
      check_launch();
      // inner reference norms ||r||^2 per RHS; inner active = outer active
      DotArgs dbi = make_dot(D->sc_in, DOT_WY, FIN_STORE_BN, nullptr, nrhs, D->nb, o.inner_tol, 0);
      launch_dot(VEC_F32, D->n_b, C, W.r, W.r, dbi, st);
      check_launch();
      launch_init_scalars(D->sc_in, nrhs, D->nb, st);
      check_launch();
      CK(cudaMemcpyAsync(D->sc_in.active, D->sc_out.active, sizeof(int32_t) * C, cudaMemcpyDeviceToDevice, st));
      launch_zero(VEC_F32, D->n_b * C, W.x, st);
      check_launch();
      const int it = pcg_loop(c, W, D->sc_in, nrhs, o.inner_tol, o.maxit - total_it, graphs,
                              0x200 | (o.precision == AMGSYM_PREC_MIXED_BF16 ? 2 : 0) | (o.finest_hat ? 1 : 0) |
                                  (o.preconditioner << 4),
                              &breakdown);
      total_it += it;
      launch_add_to_f64(VEC_F32, D->n_b * C, D->xh, W.x, st);
      check_launch();
      if (breakdown) break;
    }
  }
  if (D->singular) {
    // the minimum-norm solution: no constant component
    launch_sub_block0_mean(D->xh, D->n_b, nrhs, D->nb, D->sc_out.partials, D->sc_out.partial_cap, st);
    check_launch();
  }
  launch_transform_bwd(D->xh, VEC_F64, nrhs, D->perm, D->n_b, D->s, x_dev, ld, st);
  check_launch();
  if (breakdown) {
    CK(cudaStreamSynchronize(st));
    fail(AMGSYM_ERR_BREAKDOWN, "PCG breakdown (p^T A p <= 0 or not finite)");
  }
  const bool converged = st4[0] == 0;
  if (!converged) result = AMGSYM_NOT_CONVERGED;
  if (info) {
    CK(cudaMemcpyAsync(D->h_relres, D->sc_out.relres, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    info->iters = total_it;
    info->outer_iters = mixed ? outer : 0;
    info->converged = converged ? 1 : 0;
    if (info->relres) std::memcpy(info->relres, D->h_relres, sizeof(double) * nrhs);
  }
  return result;
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

extern "C" amgsym_status amgsym_solve(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                                      const amgsym_solve_opts* sopts, void* stream, amgsym_solve_info* info) {
  try {
    return solve_impl(h, b_dev, x_dev, nrhs, ld, sopts, stream, info);
  } catch (const amgsym::Error& e) {
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}

extern "C" amgsym_status amgsym_solve_adjoint(amgsym_t h, const double* g_dev, double* lam_dev, int32_t nrhs,
                                              int64_t ld, const amgsym_solve_opts* sopts, void* stream,
                                              amgsym_solve_info* info) {
  // A is symmetric (validated at creation), so A^T lambda = g is the same solve.
  return amgsym_solve(h, g_dev, lam_dev, nrhs, ld, sopts, stream, info);
}

extern "C" amgsym_status amgsym_transform_forward(amgsym_t h, const double* b_dev, int32_t nrhs, int64_t ld,
                                                  double* xhat_dev, void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || ld < h->n || !b_dev || !xhat_dev) fail(AMGSYM_ERR_ARG, "bad arguments");
  launch_transform_fwd(b_dev, nrhs, ld, D->perm, D->n_b, D->s, xhat_dev, VEC_F64, (cudaStream_t)stream);
  check_launch();
  API_END
}

extern "C" amgsym_status amgsym_transform_backward(amgsym_t h, const double* xhat_dev, int32_t nrhs,
                                                   double* x_dev, int64_t ld, void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || ld < h->n || !xhat_dev || !x_dev) fail(AMGSYM_ERR_ARG, "bad arguments");
  launch_transform_bwd(xhat_dev, VEC_F64, nrhs, D->perm, D->n_b, D->s, x_dev, ld, (cudaStream_t)stream);
  check_launch();
  API_END
}

extern "C" amgsym_status amgsym_apply_reduced(amgsym_t h, const void* X_dev, void* Y_dev, int32_t nrhs,
                                              int32_t prec, void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  check_ptr(X_dev, "X");
  check_ptr(Y_dev, "Y");
  if (X_dev == Y_dev) fail(AMGSYM_ERR_ARG, "X and Y must not overlap");
  const bool f64 = prec == AMGSYM_PREC_FP64;
  const VecType vt = f64 ? VEC_F64 : VEC_F32;
  const ValType mt = f64 ? VAL_F64 : VAL_F32;
  if (!D->Ainn.vals(mt)) fail(AMGSYM_ERR_STATE, "value precision not built");
  Ctx c{D, nrhs * D->nb, vt, mt, false, (cudaStream_t)stream};
  spmm(c, D->Ainn, mt, vt, vt, X_dev, Y_dev, 1.0, 0.0, nullptr, true, nullptr);
  API_END
}

extern "C" amgsym_status amgsym_vcycle(amgsym_t h, const void* R_dev, void* Z_dev, int32_t nrhs, int32_t prec,
                                       int32_t finest_hat, void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  check_ptr(R_dev, "R");
  check_ptr(Z_dev, "Z");
  if (R_dev == Z_dev) fail(AMGSYM_ERR_ARG, "R and Z must not overlap");
  const bool f64 = prec == AMGSYM_PREC_FP64;
  const VecType vt = f64 ? VEC_F64 : VEC_F32;
  const ValType mt = f64 ? VAL_F64 : prec == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : VAL_F32;
  ensure_work(D, nrhs, vt);
  Ctx c{D, nrhs * D->nb, vt, mt, finest_hat != 0, (cudaStream_t)stream};
  c.fuse = true;
  prepare_cycle(c);
  vcycle(c, 0, R_dev, Z_dev, nullptr);
  API_END
}

extern "C" amgsym_status amgsym_amgr_apply(amgsym_t h, const void* R_dev, void* Z_dev, int32_t nrhs, int32_t prec,
                                           void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (!D->has_amgr) fail(AMGSYM_ERR_STATE, "AMGR was not built: call amgsym_setup with opts.amgr = 1");
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  check_ptr(R_dev, "R");
  check_ptr(Z_dev, "Z");
  if (R_dev == Z_dev) fail(AMGSYM_ERR_ARG, "R and Z must not overlap");
  const bool f64 = prec == AMGSYM_PREC_FP64;
  const VecType vt = f64 ? VEC_F64 : VEC_F32;
  const ValType mt = f64 ? VAL_F64 : prec == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : VAL_F32;
  if (!D->Ainn.vals(mt)) fail(AMGSYM_ERR_STATE, "value precision not built");
  ensure_work(D, nrhs, vt);
  Ctx c{D, nrhs * D->nb, vt, mt, false, (cudaStream_t)stream};
  c.pc = AMGSYM_PC_AMGR;
  amgr_apply(c, R_dev, Z_dev);
  API_END
}

extern "C" amgsym_status amgsym_amgr_info(amgsym_t h, int64_t* n_coarse_per_copy, int64_t* nnz_P, int64_t* nnz_Ac,
                                          int32_t* coarse_levels, int8_t* cf) {
  API_BEGIN
  if (!h) fail(AMGSYM_ERR_ARG, "NULL handle");
  if (!h->amgr) fail(AMGSYM_ERR_STATE, "AMGR was not built: call amgsym_setup with opts.amgr = 1");
  const HostAmgr& M = *h->amgr;
  if (n_coarse_per_copy) *n_coarse_per_copy = M.n_cb;
  if (nnz_P) *nnz_P = M.Pb.nnz();
  if (nnz_Ac) *nnz_Ac = M.coarse->H.levels[0].A.nnz();
  if (coarse_levels) *coarse_levels = (int32_t)M.coarse->H.levels.size();
  if (cf) std::memcpy(cf, M.cf.data(), M.cf.size());
  API_END
}

extern "C" amgsym_status amgsym_amgr_matrix(amgsym_t h, int32_t which, int64_t* rowptr, int32_t* colidx,
                                            double* vals) {
  API_BEGIN
  if (!h || !rowptr || !colidx || !vals) fail(AMGSYM_ERR_ARG, "NULL argument");
  if (!h->amgr) fail(AMGSYM_ERR_STATE, "AMGR was not built: call amgsym_setup with opts.amgr = 1");
  if (which != 0 && which != 1) fail(AMGSYM_ERR_ARG, "which must be 0 (P_b) or 1 (A_c)");
  const Csr& M = which == 0 ? h->amgr->Pb : h->amgr->coarse->H.levels[0].A;
  std::memcpy(rowptr, M.ptr.data(), sizeof(int64_t) * M.ptr.size());
  std::memcpy(colidx, M.idx.data(), sizeof(int32_t) * M.idx.size());
  std::memcpy(vals, M.val.data(), sizeof(double) * M.val.size());
  API_END
}

extern "C" amgsym_status amgsym_cycle_timeout_check(amgsym_t h, int32_t nrhs, int32_t prec, void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  const bool f64 = prec == AMGSYM_PREC_FP64;
  const VecType vt = f64 ? VEC_F64 : VEC_F32;
  const ValType mt = f64 ? VAL_F64 : prec == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : VAL_F32;
  ensure_work(D, nrhs, vt);
  Ctx c{D, nrhs * D->nb, vt, mt, false, (cudaStream_t)stream};
  c.fuse = true;
  prepare_cycle(c);
  auto it = D->cycle_plans.find(cycle_key(c));
  if (it == D->cycle_plans.end()) fail(AMGSYM_ERR_STATE, "this problem has no persistent coarse cycle");
  const CyclePlan& pl = it->second;
  if (pl.nphases < 2) fail(AMGSYM_ERR_STATE, "the coarse cycle has no grid barrier");
  CycleBar b = D->bar;
  b.extra = 1;      // one arrival more than the grid: nothing releases the first barrier
  b.spins = 4096;   // a few milliseconds
  const cudaError_t e = launch_cycle(mt, vt, c.C, pl.grid, pl.phases, pl.nphases, b, nullptr, c.st);
  if (e != cudaSuccess) fail(AMGSYM_ERR_CUDA, std::string("coarse-cycle launch: ") + cudaGetErrorString(e));
  CK(cudaStreamSynchronize(c.st));
  int32_t err = 0;
  CK(cudaMemcpy(&err, D->bar.err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  CK(cudaMemset(D->bar.count, 0, 4 * sizeof(unsigned)));  // count, generation, error
  if (err != 1) fail(AMGSYM_ERR_CUDA, "the timed-out barrier wait was not reported");
  API_END
}

extern "C" amgsym_status amgsym_fv_grad_logk(int32_t d, const int64_t* N, const double* widths_dev,
                                             const double* k_dev, const double* u_dev, const double* lam_dev,
                                             int32_t nrhs, int64_t ld, double* grad_dev, int32_t accumulate,
                                             void* stream) {
  API_BEGIN
  if (d < 1 || d > 3 || !N) fail(AMGSYM_ERR_ARG, "grid dimension must be 1..3");
  int64_t n = 1;
  for (int a = 0; a < d; ++a) {
    if (N[a] <= 0) fail(AMGSYM_ERR_ARG, "grid extent must be positive");
    n *= N[a];
  }
  if (!widths_dev || !k_dev || !u_dev || !lam_dev || !grad_dev) fail(AMGSYM_ERR_ARG, "NULL argument");
  if (nrhs < 1 || ld < n) fail(AMGSYM_ERR_ARG, "bad nrhs / ld");
  launch_fv_grad(d, N, widths_dev, k_dev, u_dev, lam_dev, nrhs, ld, grad_dev, accumulate, (cudaStream_t)stream);
  check_launch();
  API_END
}

extern "C" int64_t amgsym_kernel_launches(void) { return amgsym::launch_count(); }

// ---------------------------------------------------------------------------
// Per-launch timing of one solve step (amgsym_profile_step).

namespace {

// Enqueue one step of solve_impl (forward transform, outer residual, PCG
// start, one PCG iteration, backward transform) with the launch hooks on.
void profile_step_body(Device* D, amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                       bool mixed, const Ctx& c, cudaStream_t st, Profiler& prof) {
  const int32_t C = c.C;
  const VecType vt = c.vt;
  Ctx c64{D, C, VEC_F64, VAL_F64, false, st};
  PrecWork& W = mixed ? D->w32 : D->w64;
  const DevScalars& sc = mixed ? D->sc_in : D->sc_out;
  const int64_t n = h->n, n_b = D->n_b;
  auto timed = [&](const std::string& kernel, const std::string& role, int64_t bytes, auto&& launch) {
    ProfScope ps(st);
    launch();
    check_launch();
    ps.end(kernel, role, -1, bytes);
  };
  prof.phase = 0;
  timed("transform_fwd_kernel<double>", "forward transform b^ = H P b", nrhs * n * 16 + n * 4,
        [&] { launch_transform_fwd(b_dev, nrhs, ld, D->perm, n_b, D->s, D->bh, VEC_F64, st); });
  DotArgs dbn = make_dot(D->sc_out, DOT_WY, FIN_STORE_BN, nullptr, nrhs, D->nb, 0.0, 0);
  timed("dot_kernel<double>", "||b^||^2", 8 * n_b * C, [&] { launch_dot(VEC_F64, n_b, C, D->bh, D->bh, dbn, st); });
  launch_init_scalars(D->sc_out, nrhs, D->nb, st);
  launch_set_value(D->sc_out.tol2, 1e-16, st);
  launch_zero(VEC_F64, n_b * C, D->xh, st);
  check_launch();
  DotArgs drr = make_dot(D->sc_out, DOT_YY, FIN_CONV, nullptr, nrhs, D->nb, 0.0, 0);
  spmm(c64, D->Ainn, VAL_F64, VEC_F64, vt, D->xh, W.r, -1.0, 1.0, D->bh, true, &drr);
  if (mixed) {
    launch_set_value(D->sc_in.tol2, 1e-16, st);
    DotArgs dbi = make_dot(D->sc_in, DOT_WY, FIN_STORE_BN, nullptr, nrhs, D->nb, 0.0, 0);
    timed("dot_kernel<float>", "||r||^2 (inner reference)", 4 * n_b * C,
          [&] { launch_dot(VEC_F32, n_b, C, W.r, W.r, dbi, st); });
    launch_init_scalars(D->sc_in, nrhs, D->nb, st);
    check_launch();
    CK(cudaMemcpyAsync(D->sc_in.active, D->sc_out.active, sizeof(int32_t) * C, cudaMemcpyDeviceToDevice, st));
    launch_zero(VEC_F32, n_b * C, W.x, st);
    check_launch();
  }
  // PCG start: z = M r with <r, z>, p = z
  DotArgs drz = make_dot(sc, DOT_WY, FIN_STORE_RZ, W.r, nrhs, D->nb, 0.0, 0);
  drz.coupled = c.pc == AMGSYM_PC_AMGR;
  precondition(c, W.r, W.z, &drz);
  timed(std::string("copy_kernel<") + tname(vt) + ">", "p = z", 2 * xsize(vt) * n_b * C,
        [&] { launch_copy(vt, n_b * C, W.p, W.z, st); });
  prof.phase = 1;
  pcg_iteration(c, W, sc, nrhs, 0.0);
  prof.phase = 0;
  if (mixed)
    timed("add_to_f64_kernel<float>", "x^ += d (refinement update)", n_b * C * (8 + 8 + 4),
          [&] { launch_add_to_f64(VEC_F32, n_b * C, D->xh, W.x, st); });
  timed("transform_bwd_kernel<double>", "backward transform x = 2^-s P H x^", nrhs * n * 16 + n * 4,
        [&] { launch_transform_bwd(D->xh, VEC_F64, nrhs, D->perm, n_b, D->s, x_dev, ld, st); });
}

}  // namespace

extern "C" amgsym_status amgsym_profile_step(amgsym_t h, const double* b_dev, double* x_dev, int32_t nrhs,
                                             int64_t ld, int32_t prec, int32_t finest_hat, int32_t preconditioner,
                                             void* stream, amgsym_prof_record* out, int32_t max_records,
                                             int32_t* count) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  if (ld < h->n || !b_dev || !x_dev) fail(AMGSYM_ERR_ARG, "bad vectors or ld");
  if (!out || !count || max_records < 1) fail(AMGSYM_ERR_ARG, "bad record buffer");
  if (prec < AMGSYM_PREC_FP64 || prec > AMGSYM_PREC_MIXED_BF16) fail(AMGSYM_ERR_ARG, "unknown precision");
  const bool mixed = prec != AMGSYM_PREC_FP64;
  const VecType vt = mixed ? VEC_F32 : VEC_F64;
  const ValType vmt = prec == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : mixed ? VAL_F32 : VAL_F64;
  if (mixed && !(h->opts.precisions & (prec == AMGSYM_PREC_MIXED_BF16 ? 4 : 2)))
    fail(AMGSYM_ERR_STATE, "setup did not build the value precision this mode needs (opts.precisions)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ensure_work(D, nrhs, vt);
  if (preconditioner != AMGSYM_PC_AMG && preconditioner != AMGSYM_PC_AMGR)
    fail(AMGSYM_ERR_ARG, "unknown preconditioner");
  if (preconditioner == AMGSYM_PC_AMGR && !D->has_amgr)
    fail(AMGSYM_ERR_STATE, "AMGR was not built (opts.amgr at setup)");
  Ctx c{D, nrhs * D->nb, vt, vmt, finest_hat != 0, st};
  c.pc = preconditioner;
  c.fuse = true;
  prepare_cycle(c);
  cudaEvent_t held = nullptr;
  CK(cudaEventCreateWithFlags(&held, cudaEventDisableTiming));
  Profiler prof;
  struct Reset {
    Profiler* p;
    cudaEvent_t e;
    ~Reset() {
      t_prof = nullptr;
      for (auto& r : p->recs) {
        if (r.e0) cudaEventDestroy(r.e0);
        if (r.e1) cudaEventDestroy(r.e1);
      }
      if (e) cudaEventDestroy(e);
    }
  } reset{&prof, held};
  // The hold kernel keeps the stream busy while the host enqueues the step,
  // so the step's kernels then run back to back and the events between them
  // time the kernels, not the host.  If the hold ran out before the last
  // launch was enqueued, try again with a longer one.
  for (int32_t naps = 300;; naps *= 2) {
    for (auto& r : prof.recs) {
      if (r.e0) cudaEventDestroy(r.e0);
      if (r.e1) cudaEventDestroy(r.e1);
    }
    prof.recs.clear();
    launch_hold(naps, st);
    check_launch();
    CK(cudaEventRecord(held, st));
    t_prof = &prof;
    profile_step_body(D, h, b_dev, x_dev, nrhs, ld, mixed, c, st, prof);
    t_prof = nullptr;
    const cudaError_t q = cudaEventQuery(held);
    CK(cudaStreamSynchronize(st));
    if (q == cudaErrorNotReady || naps >= 1600) break;
    (void)cudaGetLastError();
  }
  const int32_t nrec = (int32_t)prof.recs.size();
  for (int32_t i = 0; i < nrec && i < max_records; ++i) {
    const ProfRecord& r = prof.recs[i];
    amgsym_prof_record& o = out[i];
    std::memset(&o, 0, sizeof(o));
    std::strncpy(o.kernel, r.kernel.c_str(), sizeof(o.kernel) - 1);
    std::strncpy(o.role, r.role.c_str(), sizeof(o.role) - 1);
    o.level = r.level;
    o.phase = r.phase;
    o.bytes = r.bytes;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
    o.us = 1e3 * (double)ms;
  }
  *count = nrec;
  API_END
}

// ---------------------------------------------------------------------------
// V-cycle without allocation.
//
// amgsym_vcycle obtains its level work vectors from cudaMalloc on first use.
// Some callers cannot allow that: a real-time loop that must not take the
// device-wide synchronisation cudaMalloc/cudaFree imply, or a process whose
// device memory is entirely owned by another allocator (a framework's caching
// pool with a fixed budget), where a library-side cudaMalloc may fail or
// fragment the pool.  amgsym_vcycle_noalloc runs the same V-cycle with its
// level vectors carved from one fixed array in device global memory that the
// library declares statically; it calls no allocating routine.

namespace {

// Fixed scratch shared by every call on a device.  It exists on every GPU
// that loads this library, for the life of the process.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch for the current device.  In host code
// the symbol name is only a host-side handle, so the address is looked up
// once per device (with that device current) and cached.
void* noalloc_scratch(int dev) {
  if (dev < 0 || dev >= kMaxDevices) fail(AMGSYM_ERR_ARG, "device ordinal out of range for the no-allocation path");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) fail(AMGSYM_ERR_CUDA, "cudaGetSymbolAddress returned NULL for the no-allocation scratch");
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

// The V-cycle of vcycle() above with caller-provided level buffers.
const void* vcycle_with(const Ctx& c, std::vector<LevelWork>& lws, int l, const void* y, void* z, bool pre_done) {
  return vcycle_level(c, lws, l, y, z, nullptr, pre_done, [&](int l1, const void* y1, void* z1, bool pd) {
    return vcycle_with(c, lws, l1, y1, z1, pd);
  });
}

}  // namespace

extern "C" amgsym_status amgsym_vcycle_noalloc(amgsym_t h, const void* R_dev, void* Z_dev, int32_t nrhs,
                                               int32_t prec, int32_t finest_hat, void* stream) {
  API_BEGIN
  Device* D = require_dev(h);
  if (nrhs < 1 || (int64_t)nrhs * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
  check_ptr(R_dev, "R");
  check_ptr(Z_dev, "Z");
  if (R_dev == Z_dev) fail(AMGSYM_ERR_ARG, "R and Z must not overlap");
  const bool f64 = prec == AMGSYM_PREC_FP64;
  const VecType vt = f64 ? VEC_F64 : VEC_F32;
  const ValType mt = f64 ? VAL_F64 : prec == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : VAL_F32;
  const int32_t C = nrhs * D->nb;
  const size_t es = f64 ? 8 : 4;
  // Carve the level vectors from the fixed scratch, each 256-byte aligned:
  // y, z below the finest level (the level's right-hand side and solution);
  // r, t on every level that smooths (the dense coarsest solve reads y and
  // writes z only).
  std::vector<size_t> off;
  size_t need = 0;
  auto take = [&](int64_t rows) {
    off.push_back(need);
    need += ((size_t)rows * (size_t)C * es + 255) & ~size_t(255);
  };
  for (size_t l = 0; l < D->lv.size(); ++l) {
    const int64_t n = D->lv[l].n;
    if (!D->lv[l].cinv) {
      take(n);  // r
      take(n);  // t
    }
    if (l > 0) {
      take(n);  // y
      take(n);  // z
    }
  }
  if (need > kNoAllocScratchBytes)
    fail(AMGSYM_ERR_ARG, "amgsym_vcycle_noalloc: this problem needs " + std::to_string(need) +
                             " bytes of V-cycle scratch for nrhs = " + std::to_string(nrhs) +
                             "; the fixed scratch holds " + std::to_string(kNoAllocScratchBytes) +
                             " bytes (use amgsym_vcycle)");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  unsigned char* base = static_cast<unsigned char*>(noalloc_scratch(dev));
  std::vector<LevelWork> lws(D->lv.size());
  size_t k = 0;
  for (size_t l = 0; l < D->lv.size(); ++l) {
    if (!D->lv[l].cinv) {
      lws[l].r = base + off[k++];
      lws[l].t = base + off[k++];
    }
    if (l > 0) {
      lws[l].y = base + off[k++];
      lws[l].z = base + off[k++];
    }
  }
  Ctx c{D, C, vt, mt, finest_hat != 0, (cudaStream_t)stream};
  vcycle_with(c, lws, 0, R_dev, Z_dev, false);
  API_END
}

extern "C" amgsym_status amgsym_get_tiles(amgsym_t h, int32_t nrhs, int32_t prec, int32_t* out, int32_t max_levels) {
  API_BEGIN
  Device* D = require_dev(h);
  if (!out || max_levels < 1) fail(AMGSYM_ERR_ARG, "bad output buffer");
  const int32_t C = nrhs * D->nb;
  const bool f64 = prec == AMGSYM_PREC_FP64;
  const VecType vt = f64 ? VEC_F64 : VEC_F32;
  const ValType mt = f64 ? VAL_F64 : prec == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : VAL_F32;
  Ctx c{D, C, vt, mt, false, nullptr};
  auto put = [&](int slot, const DevCsr& M, ValType m) {
    if (!M.idx) {
      out[2 * slot] = out[2 * slot + 1] = 0;
      return;
    }
    const SpmmArgs a = make_spmm_args(c, M, m, vt, vt, nullptr, nullptr, 1.0, 0.0, nullptr, false, nullptr);
    out[2 * slot] = a.cpt;
    out[2 * slot + 1] = a.kl;
  };
  put(0, D->Ainn, f64 ? VAL_F64 : VAL_F32);
  for (int l = 0; l < max_levels; ++l) {
    const bool have = l < (int)D->lv.size() && !D->lv[l].cinv;
    const DevLevel empty;
    const DevLevel& L = have ? D->lv[l] : empty;
    put(1 + 5 * l + 0, L.A, mt);
    put(1 + 5 * l + 1, L.G, mt);
    put(1 + 5 * l + 2, L.Gt, mt);
    put(1 + 5 * l + 3, L.R, mt);
    put(1 + 5 * l + 4, L.P, mt);
  }
  API_END
}
