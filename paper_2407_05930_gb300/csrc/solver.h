// Host-side state of a problem on the device and the sequencing helpers
// shared by the single-problem solve (solve.cu) and the batched solve
// (batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "device.h"
#include "internal.h"

namespace amgsym {

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      fail(e_ == cudaErrorMemoryAllocation ? AMGSYM_ERR_OOM : AMGSYM_ERR_CUDA,            \
           std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

void check_launch();

// Precision-specific work arrays for one column count.
struct LevelWork {
  void* y = nullptr;  // level rhs (levels >= 1)
  void* z = nullptr;  // level solution (levels >= 1)
  void* r = nullptr;  // residual
  void* t = nullptr;  // smoother temporary
};

struct PrecWork {
  bool ready = false;
  std::vector<LevelWork> lw;
  void *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr;  // PCG vectors
  // AMGR V-cycle: smoother temporary and residual [n_b][C], restricted
  // residual and coarse correction [n_cb][C], the same in the coarse
  // problem's layout [n_cb * 2^s][nrhs]
  void *at = nullptr, *ar = nullptr, *arc = nullptr, *ahc = nullptr, *arc2 = nullptr, *ahc2 = nullptr;
  // AMGR coarse problem with the transformed-basis A_c (SymCoarse): the
  // operand and product in that layout [n_cb][nrhs * 2^s]
  void *sxh = nullptr, *syh = nullptr;
};

struct GraphKey {
  int mode = -1;
  int32_t nrhs = 0;
  double tol = 0.0;
  uint64_t tiles_gen = 0;  // tiles the captured launches were built with
  bool operator==(const GraphKey& o) const {
    return mode == o.mode && nrhs == o.nrhs && tol == o.tol && tiles_gen == o.tiles_gen;
  }
};

// Phases of the persistent coarse-cycle kernel for one column count,
// precision and set of work arrays (device array in the work allocations).
struct CyclePlan {
  CyclePhase* phases = nullptr;
  int32_t nphases = 0;
  int grid = 0;
};
using CycleKey = std::tuple<int32_t, int, int, uint64_t, uint64_t>;  // C, vt, mt, work_gen, tiles_gen

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
};

// SpMM tile (columns per thread, entry lanes per row) chosen by the tuner for
// one matrix, column count and precision combination.
struct Tile {
  int cpt = 0, kl = 0;
};
// matrix idx array, C, mt, xt, ot, variant (0: plain epilogue, 1: with the fused dot)
using TileKey = std::tuple<const void*, int32_t, int, int, int, int>;

// Generations come from one process-wide counter that only goes up, so a
// value identifies one Device object and one set of its work arrays for the
// life of the process: a Device created after another was freed never
// repeats its generations (a batch compares them to decide whether its plans,
// which hold device pointers, are still valid).
uint64_t next_generation();

// AMGR top level on the device (see HostAmgr): P_b, R_b = P_b^T, the FSAI of
// the inner block K (embedded, fine rows), its damping, the coarse-row
// diagonal smoother, and the coarse problem A_c with its own hierarchy.
struct DevAmgr {
  DevCsr Pb, Rb, GK, GKt;
  double omegaK = 1.0;
  double* jd64 = nullptr;
  float* jd32 = nullptr;
  int32_t n_cb = 0;
  Device* cd = nullptr;  // the coarse problem's device copy (owned by that problem)
  const void* jd(VecType t) const { return t == VEC_F64 ? (const void*)jd64 : (const void*)jd32; }
};

// The AMGR coarse operator in the transformed basis: A_c = (1 / 2^s) H
// blockdiag(A^_c,i) H with A^_c,i = Ac0 + interface couplings of block i, so
// a product with A_c (the copy layout of the coarse problem) is the butterfly
// to the transformed layout, the reduced SpMM (Ac0 read once for every block
// and right-hand side, the couplings in the interface pass), and the scaled
// butterfly back: about 1/2^s of the matrix bytes of the assembled A_c.
struct SymCoarse {
  DevCsr inn;      // Ac0 = P_b^T A_inn P_b, n_cb rows
  DevIface iface;  // coarse interface couplings, per block
  int32_t nb = 1;
  int64_t n_cb = 0;
};

struct Device {
  int device_id = 0;
  // set on the AMGR coarse problem's device: its level-0 A products run in
  // the transformed basis (opts.amgr_sym_ac of the fine problem)
  std::shared_ptr<SymCoarse> symc;
  uint64_t epoch = 0;      // next_generation() at upload: identifies this Device
  uint64_t work_gen = 0;   // next_generation() whenever work arrays are (re)allocated
  uint64_t tiles_gen = 0;  // bumped whenever the tuner changes tiles
  std::map<TileKey, Tile> tiles;
  std::set<std::tuple<int32_t, int, int>> tuned;  // (C, vt, mt) already tuned
  int precisions = 3;
  int nu = 1;
  bool singular = false;  // pure Neumann: solves remove the constant component of b and x
  int32_t s = 0, nb = 1;
  int64_t n_b = 0;
  DevCsr Ainn;  // alias of lv[0].A
  DevIface iface;
  int32_t* perm = nullptr;
  std::vector<DevLevel> lv;
  std::vector<void*> owned;  // setup allocations
  // work arrays for work_nrhs right-hand sides
  int32_t work_nrhs = 0;
  std::vector<void*> work_owned;
  double* bh = nullptr;  // b^ (FP64)
  double* xh = nullptr;  // x^ (FP64)
  PrecWork w64, w32;
  DevScalars sc_out, sc_in;
  int32_t* h_status = nullptr;  // pinned [2][4]
  double* h_relres = nullptr;   // pinned [work_nrhs]
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  GraphCache graph;
  int64_t graph_kernels = 0;
  // persistent coarse cycle: first level it runs (-1 = none), barrier words,
  // whether a cooperative launch can be captured in a graph (-1 = not probed)
  int fuse_level = -1;
  CycleBar bar;
  int coop_ok = -1;
  std::map<CycleKey, CyclePlan> cycle_plans;
  // Low-rank correction of LRCAMG(k) (eq. "LRCAMG"), per block i: the k
  // right eigenvectors U of M_inn^{-1} A^_i with the smallest eigenvalues
  // (A^_i-orthonormal) and Theta (A^_i U), both [k][n_b][nb]; Ritz values
  // theta [nb][k] (host).  lrc_k = 0: none.
  int32_t lrc_k = 0;
  double* lrc_U = nullptr;
  double* lrc_V = nullptr;
  std::vector<double> lrc_theta;
  bool has_amgr = false;
  bool zmarch = false;  // opts.zmarch: finest-level diagonal-offset products as the z-marching stencil
  DevAmgr amgr;
  // Low-rank correction of LRCFSAI(k) (eq. "LRCFSAI"), per block: Z = G_inn^T V
  // (V the k eigenvectors of G_inn A^_i G_inn^T of the smallest eigenvalues)
  // and Theta Z, both [k][n_b][nb]; Ritz values [nb][k] (host).
  int32_t lrcf_k = 0;
  double* lrcf_Z = nullptr;
  double* lrcf_TZ = nullptr;
  std::vector<double> lrcf_theta;
};

struct Ctx {
  Device* D;
  int32_t C;
  VecType vt;       // vector precision of the V-cycle / inner PCG
  ValType mt;       // matrix value precision of the V-cycle
  bool finest_hat;  // V-cycle level-0 residual with A^_i
  cudaStream_t st;
  const int32_t* skip = nullptr;  // early-exit flag (active RHS count) of the PCG loop
  bool tune = false;              // run the tile autotuner before the first PCG loop
  bool fuse = false;              // coarse levels as one persistent kernel (Device::fuse_level)
  int pc = AMGSYM_PC_AMG;         // preconditioner of the PCG: the A_inn V-cycle or AMGR
};
// The AMGR V-cycle (Alg. "apply"): z = M_AMGR y for every column of c.
void amgr_apply(const Ctx& c, const void* y, void* z);

// ---------------------------------------------------------------------------
// Per-launch timing (amgsym_profile_step): while a Profiler is installed for
// the calling thread, every instrumented launch is bracketed by two CUDA
// events on its stream and recorded with its kernel, its role in the solve
// and its algorithmic bytes.  Without one the hooks cost a thread-local load.
struct ProfRecord {
  std::string kernel, role;
  int32_t level = -1, phase = 0;
  int64_t bytes = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};
struct Profiler {
  std::vector<ProfRecord> recs;
  int32_t phase = 0;  // 0: once per solve / refinement step, 1: every PCG iteration
};
extern thread_local Profiler* t_prof;
class ProfScope {
 public:
  explicit ProfScope(cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;
  bool on() const { return ev0_ != nullptr; }
  void end(const std::string& kernel, const std::string& role, int level, int64_t bytes);

 private:
  cudaStream_t st_;
  cudaEvent_t ev0_ = nullptr;
};

// Build (outside graph capture) the persistent coarse-cycle plan the V-cycle
// of this context will use, and check the barrier error word after a run.
void prepare_cycle(const Ctx& c);
void check_cycle_error(Device* D, cudaStream_t st);


void ensure_work(Device* D, int32_t nrhs, VecType vt);
// One V-cycle of the A_inn hierarchy: Z = (I (x) M_inn^{-1}) R (amgsym_vcycle).
void vcycle_apply(const Ctx& c, const void* R, void* Z);
void tune_tiles(const Ctx& c);
Tile fixed_tile(const DevCsr& M, int32_t C, VecType xt);
SpmmArgs make_spmm_args(const Ctx& c, const DevCsr& M, ValType mt, VecType xt, VecType ot, const void* X,
                        void* Y, double alpha, double beta, const void* Z, bool iface, const DotArgs* dot);
void spmm(const Ctx& c, const DevCsr& M, ValType mt, VecType xt, VecType ot, const void* X, void* Y, double alpha,
          double beta, const void* Z, bool iface, const DotArgs* dot);
DotArgs make_dot(const DevScalars& sc, int mode, int final, const void* W, int32_t nrhs, int32_t nb, double tol,
                 int count_iter);
Device* require_dev(amgsym_t h);
void check_ptr(const void* p, const char* what);

}  // namespace amgsym
