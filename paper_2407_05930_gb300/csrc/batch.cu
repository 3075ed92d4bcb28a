// Batched solve: many independent problems (uneven sizes, symmetry counts and
// RHS counts) advance through the same mixed-precision refinement and inner
// PCG in lock step.  Every step of an inner PCG iteration -- the reduced
// SpMM, the vector updates, each smoother / residual / restriction /
// prolongation product of every V-cycle level and the coarsest solves -- is
// one persistent work-list launch over all problems that take part in it
// (k_batch.cu), and one iteration is captured in a CUDA graph and replayed.
// Problems whose hierarchy ends at a level do their coarsest solve there while
// deeper problems continue down, so hierarchies of different depth share the
// launches level by level.  Tiles (columns per thread, entry lanes per row)
// come from each problem's autotuner run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "device.h"
#include "dot.cuh"
#include "internal.h"
#include "solver.h"

namespace amgsym {

struct BLaunch {
  int kind = 0;  // 0 SpMM, 1 vector op, 2 coarse
  ValType mt = VAL_F32;
  VecType xt = VEC_F32, ot = VEC_F32;
  int cpt = 4, kl = 1, op = 0;
  bool dot = false, ifc = false, dia = false;
  void* args = nullptr;
  BItem* items = nullptr;
  BDot* dots = nullptr;
  int32_t n_items = 0;
  size_t smem = 0;
};

struct Batch {
  std::vector<amgsym_t> probs;
  std::vector<int32_t> nrhs, C;
  int count = 0;
  int device_id = 0;
  std::vector<void*> owned;       // status / tolerance arrays
  std::vector<void*> plan_owned;  // plan arrays (rebuilt per precision)
  int32_t* status_in = nullptr;   // [count][4]
  int32_t* status_out = nullptr;  // [count][4]
  double* tol2_in = nullptr;      // [count]
  double* tol2_out = nullptr;     // [count]
  int32_t* h_status = nullptr;    // pinned [2][count][4]
  double* h_tol2 = nullptr;       // pinned [count]
  double* h_relres = nullptr;     // pinned [sum nrhs]
  std::vector<DevScalars> sc_in, sc_out;
  std::vector<BLaunch> plan_iter, plan_start, plan_resid;
  int planned_key = -1;
  // (Device epoch, work generation) of every problem when the plans were
  // built: the plans and the graph hold that Device's matrix and work
  // pointers, which amgsym_update_values / amgsym_setup free
  std::vector<uint64_t> planned_gen;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_kernels = 0;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // batched autotuner: on while plans are built with sopts->tune = 1
  bool tune = false;
  cudaStream_t tune_stream = nullptr;
  std::map<std::vector<const void*>, std::pair<int, int>> tuned;  // matrices of a step -> (cpt, kl)
};

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      fail(e_ == cudaErrorMemoryAllocation ? AMGSYM_ERR_OOM : AMGSYM_ERR_CUDA,             \
           std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

template <typename T>
static T* bupload(std::vector<void*>& owner, const std::vector<T>& v) {
  if (v.empty()) return nullptr;
  void* p = nullptr;
  BCK(cudaMalloc(&p, sizeof(T) * v.size()));
  owner.push_back(p);
  BCK(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return static_cast<T*>(p);
}

// Dot scratch of one (launch, problem): partials, chunk partials and zeroed
// tickets for the two-level reduction of block_dot2.
static BDot alloc_bdot(Batch* B, int32_t nslots, int32_t C) {
  BDot bd;
  const int32_t nch = (nslots + 31) / 32;
  void* p = nullptr;
  BCK(cudaMalloc(&p, sizeof(double) * (size_t)nslots * C));
  B->plan_owned.push_back(p);
  bd.partials = static_cast<double*>(p);
  BCK(cudaMalloc(&p, sizeof(double) * (size_t)nch * C));
  B->plan_owned.push_back(p);
  bd.chunk_partials = static_cast<double*>(p);
  BCK(cudaMalloc(&p, sizeof(unsigned) * (size_t)(nch + 1)));
  B->plan_owned.push_back(p);
  BCK(cudaMemset(p, 0, sizeof(unsigned) * (size_t)(nch + 1)));
  bd.chunk_tickets = static_cast<unsigned*>(p);
  bd.ticket = bd.chunk_tickets + nch;
  bd.nslots = nslots;
  return bd;
}

static void free_plans(Batch* B) {
  for (void* p : B->plan_owned) cudaFree(p);
  B->plan_owned.clear();
  B->plan_iter.clear();
  B->plan_start.clear();
  B->plan_resid.clear();
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->graph = nullptr;
  B->planned_key = -1;
}

// Rows per item (in row slots of rows_pb rows): sized so that one wave of
// resident blocks touches about 48 MB of the gathered vector (row_bytes per
// row).  The far-neighbour rows a block gathers are then still in L2 from the
// blocks working just behind it, even when the vector is larger than L2.
static int slots_per_item(int64_t rows, int rows_pb, int64_t row_bytes) {
  (void)rows;
  const int64_t wave = (int64_t)max_grid_blocks();
  const int64_t rows_item = std::max<int64_t>(rows_pb, (int64_t(48) << 20) / (wave * std::max<int64_t>(row_bytes, 1)));
  return (int)std::max<int64_t>(1, std::min<int64_t>(rows_item / rows_pb, 4096 / rows_pb));
}

// Resolved tile of one SpMM argument record (as the launcher would pick it).
static void resolve_tile(const SpmmArgs& a, VecType xt, VecType ot, int* cpt, int* kl) {
  const int es = std::max(xt == VEC_F64 ? 8 : 4, ot == VEC_F64 ? 8 : 4);
  const int V = 16 / es;
  int c = a.cpt > 0 ? a.cpt : V;
  if (c >= 2 * V && a.C % (2 * V) == 0 && a.C / (2 * V) <= kBlock)
    c = 2 * V;
  else if (a.C % V == 0 && a.C / V <= kBlock)
    c = V;
  else if (V >= 2 && a.C % 2 == 0)
    c = 2;
  else
    c = 1;
  if (xt == VEC_F64 || ot == VEC_F64) c = std::min(c, xt == VEC_F64 && ot == VEC_F64 ? 4 : 2);
  const int tpc = a.C / c;
  int k = a.kl > 0 ? a.kl : 1;
  if ((tpc & (tpc - 1)) || a.ndiag > 0) k = 1;
  while (k > 1 && tpc * k > 32) k >>= 1;
  *cpt = c;
  *kl = k;
}

static void run_plan(const std::vector<BLaunch>& plan, cudaStream_t st);

// One batched SpMM step: args[p] for each taking part problem (DotArgs inside).
// Device arrays of the launches go to `owner`.
static void add_spmm_core(Batch* B, std::vector<BLaunch>& plan, const std::vector<SpmmArgs>& args, ValType mt,
                          VecType xt, VecType ot, std::vector<void*>& owner) {
  std::map<std::tuple<int, int, bool, bool, bool>, std::vector<int>> groups;
  std::vector<int> cpts(args.size()), kls(args.size());
  for (size_t i = 0; i < args.size(); ++i) {
    resolve_tile(args[i], xt, ot, &cpts[i], &kls[i]);
    groups[std::make_tuple(cpts[i], kls[i], args[i].dot.mode != DOT_NONE, args[i].imask != nullptr,
                           args[i].ndiag > 0)]
        .push_back((int)i);
  }
  for (auto& kv : groups) {
    BLaunch L;
    L.kind = 0;
    L.mt = mt;
    L.xt = xt;
    L.ot = ot;
    std::tie(L.cpt, L.kl, L.dot, L.ifc, L.dia) = kv.first;
    std::vector<SpmmArgs> ga;
    std::vector<BItem> items;
    std::vector<BDot> dots;
    size_t smem_d = 0;
    for (int i : kv.second) {
      const SpmmArgs& a = args[i];
      const int arg = (int)ga.size();
      ga.push_back(a);
      const int S = (a.C / L.cpt) * L.kl;
      const int rows_pb = kBlock / S;
      const int m = slots_per_item(a.rows, rows_pb, (int64_t)a.C * (xt == VEC_F64 ? 8 : 4));
      const int64_t slots = ((int64_t)a.rows + rows_pb - 1) / rows_pb;
      int32_t slot = 0;
      for (int64_t s0 = 0; s0 < slots; s0 += m, ++slot) {
        BItem it;
        it.arg = arg;
        it.first_slot = (int32_t)s0;
        it.row_end = (int32_t)std::min<int64_t>(a.rows, (s0 + m) * rows_pb);
        it.slot = slot;
        items.push_back(it);
      }
      BDot bd;
      if (L.dot) {
        bd = alloc_bdot(B, slot, a.C);
        smem_d = std::max(smem_d, sizeof(double) * (size_t)dot_smem_doubles(S, rows_pb, a.C));
      }
      dots.push_back(bd);
    }
    // items stay in row order problem by problem: a wave of blocks then
    // sweeps contiguous row windows, so far-neighbour gathers hit L2
    std::vector<BItem> mixed = items;
    L.args = bupload(owner, ga);
    L.items = bupload(owner, mixed);
    L.dots = bupload(owner, dots);
    L.n_items = (int32_t)mixed.size();
    L.smem = smem_d;
    plan.push_back(L);
  }
}

// The batched autotuner: for a step without fused dots, time the whole
// batched step (every problem taking part) under each candidate tile --
// columns per thread (one or two 16-byte vectors) x entry lanes (1..16),
// clamped per problem to what its column count allows -- and keep the
// fastest.  Steps over the same matrices (pre- and post-smoothing) share the
// choice.  Timing runs the real work arrays (their contents do not matter).
static void add_spmm(Batch* B, std::vector<BLaunch>& plan, std::vector<SpmmArgs> args, ValType mt, VecType xt,
                     VecType ot) {
  bool dot = false;
  for (const SpmmArgs& a : args) dot = dot || a.dot.mode != DOT_NONE;
  if (B->tune && !dot && !args.empty()) {
    std::vector<const void*> key;
    for (const SpmmArgs& a : args) key.push_back(a.idx);
    auto it = B->tuned.find(key);
    if (it == B->tuned.end()) {
      const int V = (xt == VEC_F64 || ot == VEC_F64) ? 2 : 4;
      cudaEvent_t e0, e1;
      BCK(cudaEventCreate(&e0));
      BCK(cudaEventCreate(&e1));
      float best_ms = 1e30f;
      std::pair<int, int> best(0, 0);
      bool all_dia = true;  // entry lanes do not apply to the diagonal-offset form
      for (const SpmmArgs& a : args) all_dia = all_dia && a.ndiag > 0;
      for (int cm = 1; cm <= 2; ++cm)
        for (int kl = 1; kl <= (all_dia ? 1 : 16); kl *= 2) {
          std::vector<SpmmArgs> cand = args;
          for (SpmmArgs& a : cand) {
            a.cpt = V * cm;
            a.kl = kl;
          }
          std::vector<BLaunch> tmp;
          std::vector<void*> tmp_owned;
          add_spmm_core(B, tmp, cand, mt, xt, ot, tmp_owned);
          run_plan(tmp, B->tune_stream);  // warm-up
          BCK(cudaEventRecord(e0, B->tune_stream));
          for (int r = 0; r < 3; ++r) run_plan(tmp, B->tune_stream);
          BCK(cudaEventRecord(e1, B->tune_stream));
          BCK(cudaEventSynchronize(e1));
          float ms = 0.f;
          BCK(cudaEventElapsedTime(&ms, e0, e1));
          for (void* q : tmp_owned) cudaFree(q);
          if (ms < best_ms * 0.97f) {
            best_ms = ms;
            best = {V * cm, kl};
          }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      it = B->tuned.emplace(key, best).first;
    }
    for (SpmmArgs& a : args) {
      a.cpt = it->second.first;
      a.kl = it->second.second;
    }
  }
  add_spmm_core(B, plan, args, mt, xt, ot, B->plan_owned);
}

static void add_vec(Batch* B, std::vector<BLaunch>& plan, int op, VecType vt, const std::vector<UpdArgs>& args) {
  if (args.empty()) return;
  BLaunch L;
  L.kind = 1;
  L.op = op;
  L.xt = vt;
  const int V = vt == VEC_F64 ? 2 : 4;
  int cpt = V;
  for (const UpdArgs& a : args)
    if (a.C % cpt) cpt = 1;
  L.cpt = cpt;
  std::vector<BItem> items;
  std::vector<BDot> dots;
  size_t smem_d = 0;
  for (size_t i = 0; i < args.size(); ++i) {
    const UpdArgs& a = args[i];
    const int tpr = a.C / cpt;
    const int rows_pb = kBlock / tpr;
    const int m = slots_per_item(a.rows, rows_pb, (int64_t)a.C * (vt == VEC_F64 ? 8 : 4));
    const int64_t slots = ((int64_t)a.rows + rows_pb - 1) / rows_pb;
    int32_t slot = 0;
    for (int64_t s0 = 0; s0 < slots; s0 += m, ++slot) {
      BItem it;
      it.arg = (int32_t)i;
      it.first_slot = (int32_t)s0;
      it.row_end = (int32_t)std::min<int64_t>(a.rows, (s0 + m) * rows_pb);
      it.slot = slot;
      items.push_back(it);
    }
    BDot bd;
    if (op == BOP_UPDATE1) {
      bd = alloc_bdot(B, slot, a.C);
      smem_d = std::max(smem_d, sizeof(double) * (size_t)dot_smem_doubles(tpr, rows_pb, a.C));
    }
    dots.push_back(bd);
  }
  std::vector<BItem> mixed = items;
  L.args = bupload(B->plan_owned, args);
  L.items = bupload(B->plan_owned, mixed);
  L.dots = bupload(B->plan_owned, dots);
  L.n_items = (int32_t)mixed.size();
  L.smem = smem_d;
  plan.push_back(L);
}

static void add_coarse(Batch* B, std::vector<BLaunch>& plan, VecType vt, const std::vector<CoarseArgs>& args) {
  if (args.empty()) return;
  BLaunch L;
  L.kind = 2;
  L.xt = vt;
  std::vector<BItem> items;
  for (size_t i = 0; i < args.size(); ++i)
    for (int r = 0; r < args[i].n; r += 32) {
      BItem it;
      it.arg = (int32_t)i;
      it.first_slot = r;
      it.row_end = std::min(args[i].n, r + 32);
      it.slot = 0;
      items.push_back(it);
    }
  L.args = bupload(B->plan_owned, args);
  L.items = bupload(B->plan_owned, items);
  L.n_items = (int32_t)items.size();
  plan.push_back(L);
}

static void run_plan(const std::vector<BLaunch>& plan, cudaStream_t st) {
  for (const BLaunch& L : plan) {
    if (L.kind == 0)
      launch_spmm_batch(L.mt, L.xt, L.ot, L.cpt, L.kl, L.dot, L.ifc, L.dia, static_cast<const SpmmArgs*>(L.args), L.items,
                        L.n_items, L.dots, L.smem, st);
    else if (L.kind == 1)
      launch_vec_batch(L.op, L.xt, L.cpt, static_cast<const UpdArgs*>(L.args), L.items, L.n_items, L.dots, L.smem,
                       st);
    else
      launch_coarse_batch(L.xt, static_cast<const CoarseArgs*>(L.args), L.items, L.n_items, st);
    check_launch();
  }
}

// Level-synchronous V-cycle over the problems in `ps` (indices into the batch)
// at level l: y[k] -> z[k] for problem ps[k].  `last` (level 0 only) are the
// fused dots of the final smoothing product, one per problem of ps.
static void plan_vcycle(Batch* B, std::vector<BLaunch>& plan, std::vector<Ctx>& ctx, int l, const std::vector<int>& ps,
                        const std::vector<const void*>& y, const std::vector<void*>& z,
                        const std::vector<DotArgs>* last) {
  std::vector<CoarseArgs> coarse;
  std::vector<int> deep;
  std::vector<const void*> dy;
  std::vector<void*> dz;
  std::vector<DotArgs> dlast;
  for (size_t k = 0; k < ps.size(); ++k) {
    const Ctx& c = ctx[ps[k]];
    const DevLevel& L = c.D->lv[l];
    if (L.cinv) {
      if (last) fail(AMGSYM_ERR_STATE, "batched solve needs at least two levels per problem");
      CoarseArgs a;
      a.n = L.n;
      a.C = c.C;
      a.Ainv = L.cinv;
      a.Y = y[k];
      a.Z = z[k];
      a.skip = c.skip;
      coarse.push_back(a);
    } else {
      deep.push_back(ps[k]);
      dy.push_back(y[k]);
      dz.push_back(z[k]);
      if (last) dlast.push_back((*last)[k]);
    }
  }
  add_coarse(B, plan, ctx[0].vt, coarse);
  if (deep.empty()) return;
  auto lw = [&](int p) -> LevelWork& {
    Device* D = ctx[p].D;
    return (ctx[p].vt == VEC_F64 ? D->w64 : D->w32).lw[l];
  };
  auto cw = [&](int p) -> LevelWork& {
    Device* D = ctx[p].D;
    return (ctx[p].vt == VEC_F64 ? D->w64 : D->w32).lw[l + 1];
  };
  const VecType vt = ctx[0].vt;
  const ValType mt = ctx[0].mt;
  auto phase = [&](auto make) {
    std::vector<SpmmArgs> v;
    for (size_t k = 0; k < deep.size(); ++k) v.push_back(make(k, deep[k]));
    add_spmm(B, plan, v, mt, vt, vt);
  };
  auto L_ = [&](int p) -> const DevLevel& { return ctx[p].D->lv[l]; };
  const int nu = ctx[deep[0]].D->nu;
  // Smoother steps as smooth_first / smooth_sweep of the single-problem
  // V-cycle: a problem whose G_l is diagonal takes one elementwise step, the
  // others the two FSAI products (the one carrying a fused dot always does).
  auto smooth = [&](bool first, bool fin) {
    std::vector<UpdArgs> jac;
    std::vector<SpmmArgs> g, gt;
    for (size_t k = 0; k < deep.size(); ++k) {
      const int p = deep[k];
      const void* jd = L_(p).jd(vt);
      if (jd && !fin) {
        UpdArgs a;
        a.rows = L_(p).n;
        a.C = ctx[p].C;
        a.x = dz[k];
        a.p = first ? dy[k] : lw(p).r;
        a.jd = jd;
        a.accumulate = first ? 0 : 1;
        a.skip = ctx[p].skip;
        jac.push_back(a);
      } else {
        g.push_back(make_spmm_args(ctx[p], L_(p).G, mt, vt, vt, first ? dy[k] : lw(p).r, lw(p).t, 1.0, 0.0, nullptr,
                                   false, nullptr));
        gt.push_back(make_spmm_args(ctx[p], L_(p).Gt, mt, vt, vt, lw(p).t, dz[k], L_(p).omega, first ? 0.0 : 1.0,
                                    first ? nullptr : dz[k], false, fin ? &dlast[k] : nullptr));
      }
    }
    add_vec(B, plan, BOP_JACOBI, vt, jac);
    if (!g.empty()) {
      add_spmm(B, plan, g, mt, vt, vt);
      add_spmm(B, plan, gt, mt, vt, vt);
    }
  };
  // presmoothing from zero, extra sweeps, residual, restriction
  smooth(true, false);
  for (int s = 1; s < nu; ++s) {
    phase([&](size_t k, int p) { return make_spmm_args(ctx[p], L_(p).A, mt, vt, vt, dz[k], lw(p).r, -1.0, 1.0, dy[k], ctx[p].finest_hat && l == 0, nullptr); });
    smooth(false, false);
  }
  phase([&](size_t k, int p) { return make_spmm_args(ctx[p], L_(p).A, mt, vt, vt, dz[k], lw(p).r, -1.0, 1.0, dy[k], ctx[p].finest_hat && l == 0, nullptr); });
  phase([&](size_t k, int p) { return make_spmm_args(ctx[p], L_(p).R, mt, vt, vt, lw(p).r, cw(p).y, 1.0, 0.0, nullptr, false, nullptr); });
  {
    std::vector<const void*> ny;
    std::vector<void*> nz;
    for (int p : deep) {
      ny.push_back(cw(p).y);
      nz.push_back(cw(p).z);
    }
    plan_vcycle(B, plan, ctx, l + 1, deep, ny, nz, nullptr);
  }
  phase([&](size_t k, int p) { return make_spmm_args(ctx[p], L_(p).P, mt, vt, vt, cw(p).z, dz[k], 1.0, 1.0, dz[k], false, nullptr); });
  for (int s = 0; s < nu; ++s) {
    const bool fin = (s == nu - 1) && last;
    phase([&](size_t k, int p) { return make_spmm_args(ctx[p], L_(p).A, mt, vt, vt, dz[k], lw(p).r, -1.0, 1.0, dy[k], ctx[p].finest_hat && l == 0, nullptr); });
    smooth(false, fin);
  }
}

static void build_plans(Batch* B, std::vector<Ctx>& ctx, int key) {
  free_plans(B);
  const int n = B->count;
  std::vector<int> all(n);
  for (int p = 0; p < n; ++p) all[p] = p;
  const VecType vt = ctx[0].vt;
  const ValType kmt = vt == VEC_F64 ? VAL_F64 : VAL_F32;
  auto W = [&](int p) -> PrecWork& { return vt == VEC_F64 ? ctx[p].D->w64 : ctx[p].D->w32; };
  // outer FP64 residual r32 = float(b^ - A^ x^) with the outer convergence test
  {
    std::vector<SpmmArgs> v;
    for (int p = 0; p < n; ++p) {
      Ctx c64 = ctx[p];
      c64.skip = nullptr;
      DotArgs drr = make_dot(B->sc_out[p], DOT_YY, FIN_CONV, nullptr, B->nrhs[p], ctx[p].D->nb, 0.0, 0);
      v.push_back(make_spmm_args(c64, ctx[p].D->Ainn, VAL_F64, VEC_F64, vt, ctx[p].D->xh, W(p).r, -1.0, 1.0,
                                 ctx[p].D->bh, true, &drr));
    }
    add_spmm(B, B->plan_resid, v, VAL_F64, VEC_F64, vt);
  }
  // start of the inner PCG: z = M r (rz), p = z
  {
    std::vector<const void*> y;
    std::vector<void*> z;
    std::vector<DotArgs> last;
    for (int p = 0; p < n; ++p) {
      y.push_back(W(p).r);
      z.push_back(W(p).z);
      last.push_back(make_dot(B->sc_in[p], DOT_WY, FIN_STORE_RZ, W(p).r, B->nrhs[p], ctx[p].D->nb, 0.0, 0));
    }
    plan_vcycle(B, B->plan_start, ctx, 0, all, y, z, &last);
    std::vector<UpdArgs> cp;
    for (int p = 0; p < n; ++p) {
      UpdArgs u;
      u.rows = (int32_t)ctx[p].D->n_b;
      u.C = ctx[p].C;
      u.x = W(p).p;
      u.p = W(p).z;
      u.skip = ctx[p].skip;
      cp.push_back(u);
    }
    add_vec(B, B->plan_start, BOP_COPY, vt, cp);
  }
  // one PCG iteration
  {
    std::vector<SpmmArgs> k3;
    for (int p = 0; p < n; ++p) {
      DotArgs dpq = make_dot(B->sc_in[p], DOT_WY, FIN_ALPHA, W(p).p, B->nrhs[p], ctx[p].D->nb, 0.0, 0);
      k3.push_back(make_spmm_args(ctx[p], ctx[p].D->Ainn, kmt, vt, vt, W(p).p, W(p).q, 1.0, 0.0, nullptr, true, &dpq));
    }
    add_spmm(B, B->plan_iter, k3, kmt, vt, vt);
    std::vector<UpdArgs> u1;
    for (int p = 0; p < n; ++p) {
      UpdArgs u;
      u.rows = (int32_t)ctx[p].D->n_b;
      u.C = ctx[p].C;
      u.x = W(p).x;
      u.r = W(p).r;
      u.p = W(p).p;
      u.q = W(p).q;
      u.skip = ctx[p].skip;
      u.dot = make_dot(B->sc_in[p], DOT_YY, FIN_CONV, nullptr, B->nrhs[p], ctx[p].D->nb, 0.0, 1);
      u1.push_back(u);
    }
    add_vec(B, B->plan_iter, BOP_UPDATE1, vt, u1);
    std::vector<const void*> y;
    std::vector<void*> z;
    std::vector<DotArgs> last;
    for (int p = 0; p < n; ++p) {
      y.push_back(W(p).r);
      z.push_back(W(p).z);
      last.push_back(make_dot(B->sc_in[p], DOT_WY, FIN_BETA, W(p).r, B->nrhs[p], ctx[p].D->nb, 0.0, 0));
    }
    plan_vcycle(B, B->plan_iter, ctx, 0, all, y, z, &last);
    std::vector<UpdArgs> u2;
    for (int p = 0; p < n; ++p) {
      UpdArgs u;
      u.rows = (int32_t)ctx[p].D->n_b;
      u.C = ctx[p].C;
      u.x = W(p).p;
      u.p = W(p).z;
      u.beta = B->sc_in[p].beta;
      u.skip = ctx[p].skip;
      u2.push_back(u);
    }
    add_vec(B, B->plan_iter, BOP_UPDATE2, vt, u2);
  }
  B->planned_key = key;
}

static void batch_free(Batch* B) {
  if (!B) return;
  cudaSetDevice(B->device_id);
  cudaDeviceSynchronize();
  free_plans(B);
  for (void* p : B->owned) cudaFree(p);
  if (B->h_status) cudaFreeHost(B->h_status);
  if (B->h_tol2) cudaFreeHost(B->h_tol2);
  if (B->h_relres) cudaFreeHost(B->h_relres);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  if (B->tune_stream) cudaStreamDestroy(B->tune_stream);
  for (auto& e : B->ev)
    if (e) cudaEventDestroy(e);
  delete B;
}

static amgsym_status batch_solve_impl(Batch* B, const double* const* b_dev, double* const* x_dev,
                                      const amgsym_solve_opts* sopts, void* stream, amgsym_solve_info* infos) {
  amgsym_solve_opts o;
  amgsym_solve_opts_default(&o);
  if (sopts) o = *sopts;
  if (o.precision == AMGSYM_PREC_FP64)
    fail(AMGSYM_ERR_ARG, "the batched solve runs the mixed-precision refinement (AMGSYM_PREC_MIXED_*)");
  if (!(o.tol > 0.0) || o.maxit < 1) fail(AMGSYM_ERR_ARG, "bad tolerance or maxit");
  if (!b_dev || !x_dev) fail(AMGSYM_ERR_ARG, "NULL vector arrays");
  BCK(cudaSetDevice(B->device_id));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = B->count;
  const VecType vt = VEC_F32;
  const ValType vmt = o.precision == AMGSYM_PREC_MIXED_BF16 ? VAL_BF16 : VAL_F32;
  std::vector<Ctx> ctx(n);
  for (int p = 0; p < n; ++p) {
    Device* D = require_dev(B->probs[p]);
    // the conditions of amgsym_batch_create, again: a problem may have been
    // set up anew since (amgsym_update_values + amgsym_setup)
    if (D->device_id != B->device_id)
      fail(AMGSYM_ERR_STATE, "problem " + std::to_string(p) + " is no longer on the batch's device");
    if (D->lv.size() < 2)
      fail(AMGSYM_ERR_STATE, "problem " + std::to_string(p) + " now has a single-level hierarchy");
    if (D->singular) fail(AMGSYM_ERR_STATE, "problem " + std::to_string(p) + " is now singular (pure Neumann)");
    if (D->nu != require_dev(B->probs[0])->nu)
      fail(AMGSYM_ERR_STATE, "the problems of a batch must use the same nu");
    BCK(cudaSetDevice(B->device_id));
    if (!b_dev[p] || !x_dev[p]) fail(AMGSYM_ERR_ARG, "NULL vector for problem " + std::to_string(p));
    if (!(B->probs[p]->opts.precisions & (vmt == VAL_BF16 ? 4 : 2)))
      fail(AMGSYM_ERR_STATE, "problem " + std::to_string(p) + " was set up without the value precision of this mode");
    ensure_work(D, B->nrhs[p], vt);
    ctx[p] = Ctx{D, B->C[p], vt, vmt, o.finest_hat != 0, st};
    ctx[p].skip = B->status_in + 4 * p;
  }
  BCK(cudaSetDevice(B->device_id));
  // per-problem scalars with the status and tolerance redirected into the
  // batch's contiguous arrays (one copy per check for all problems)
  B->sc_in.resize(n);
  B->sc_out.resize(n);
  for (int p = 0; p < n; ++p) {
    B->sc_in[p] = ctx[p].D->sc_in;
    B->sc_in[p].status = B->status_in + 4 * p;
    B->sc_in[p].tol2 = B->tol2_in + p;
    B->sc_out[p] = ctx[p].D->sc_out;
    B->sc_out[p].status = B->status_out + 4 * p;
    B->sc_out[p].tol2 = B->tol2_out + p;
  }
  const int key = (vmt == VAL_BF16 ? 2 : 1) | (o.finest_hat ? 4 : 0);
  auto generations = [&]() {
    std::vector<uint64_t> g(2 * (size_t)n);
    for (int p = 0; p < n; ++p) {
      g[2 * p] = ctx[p].D->epoch;
      g[2 * p + 1] = ctx[p].D->work_gen;
    }
    return g;
  };
  if (B->planned_key != key || B->planned_gen != generations()) {
    B->tune = o.tune != 0;
    B->tuned.clear();
    BCK(cudaStreamSynchronize(st));  // no earlier work of this batch in flight
    if (B->tune) {
      // the timed steps must not skip: mark every problem active meanwhile
      std::vector<int32_t> act(4 * n, 0);
      for (int p = 0; p < n; ++p) act[4 * p] = 1;
      BCK(cudaMemcpy(B->status_in, act.data(), sizeof(int32_t) * 4 * n, cudaMemcpyHostToDevice));
    }
    build_plans(B, ctx, key);
    if (B->tune) {
      BCK(cudaStreamSynchronize(B->tune_stream));
      BCK(cudaMemset(B->status_in, 0, sizeof(int32_t) * 4 * n));
      B->tune = false;
    }
    B->planned_gen = generations();  // tuning allocates nothing, but be exact
  }
  // forward transforms, norms, initial state (per problem; outside the loop)
  for (int p = 0; p < n; ++p) {
    Device* D = ctx[p].D;
    amgsym_problem* P = B->probs[p];
    launch_transform_fwd(b_dev[p], B->nrhs[p], P->n, D->perm, D->n_b, D->s, D->bh, VEC_F64, st);
    DotArgs dbn = make_dot(B->sc_out[p], DOT_WY, FIN_STORE_BN, nullptr, B->nrhs[p], D->nb, o.tol, 0);
    launch_dot(VEC_F64, D->n_b, B->C[p], D->bh, D->bh, dbn, st);
    launch_init_scalars(B->sc_out[p], B->nrhs[p], D->nb, st);
    launch_set_value(B->sc_out[p].tol2, o.tol * o.tol, st);
    launch_zero(VEC_F64, D->n_b * B->C[p], D->xh, st);
    check_launch();
  }
  int total_it = 0, outer = 0;
  bool breakdown = false;
  int64_t relres_off_total = 0;
  for (int p = 0; p < n; ++p) relres_off_total += B->nrhs[p];
  auto read_out = [&](int32_t* any_active) {
    BCK(cudaMemcpyAsync(B->h_status, B->status_out, sizeof(int32_t) * 4 * n, cudaMemcpyDeviceToHost, st));
    int64_t off = 0;
    for (int p = 0; p < n; ++p) {
      BCK(cudaMemcpyAsync(B->h_relres + off, B->sc_out[p].relres, sizeof(double) * B->nrhs[p], cudaMemcpyDeviceToHost, st));
      off += B->nrhs[p];
    }
    BCK(cudaStreamSynchronize(st));
    int32_t a = 0;
    for (int p = 0; p < n; ++p) a += B->h_status[4 * p];
    *any_active = a;
  };
  int32_t active_out = 0;
  for (outer = 0; outer <= o.max_outer; ++outer) {
    run_plan(B->plan_resid, st);
    read_out(&active_out);
    if (active_out == 0 || outer == o.max_outer || total_it >= o.maxit) break;
    // per-problem inner targets (as in the single-problem refinement)
    int64_t off = 0;
    for (int p = 0; p < n; ++p) {
      double worst = 0.0;
      for (int r = 0; r < B->nrhs[p]; ++r) worst = std::max(worst, B->h_relres[off + r]);
      off += B->nrhs[p];
      double eta = worst > 0.0 ? 0.25 * o.tol / worst : o.inner_tol;
      eta = std::min(0.5, std::max(o.inner_tol, eta));
      B->h_tol2[p] = eta * eta;
    }
    BCK(cudaMemcpyAsync(B->tol2_in, B->h_tol2, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    for (int p = 0; p < n; ++p) {
      Device* D = ctx[p].D;
      PrecWork& W = D->w32;
      DotArgs dbi = make_dot(B->sc_in[p], DOT_WY, FIN_STORE_BN, nullptr, B->nrhs[p], D->nb, o.inner_tol, 0);
      launch_dot(VEC_F32, D->n_b, B->C[p], W.r, W.r, dbi, st);
      launch_init_scalars(B->sc_in[p], B->nrhs[p], D->nb, st);
      BCK(cudaMemcpyAsync(B->sc_in[p].active, B->sc_out[p].active, sizeof(int32_t) * B->C[p], cudaMemcpyDeviceToDevice, st));
      launch_zero(VEC_F32, D->n_b * B->C[p], W.x, st);
      check_launch();
    }
    // inner PCG, all problems in lock step
    run_plan(B->plan_start, st);
    if (o.use_graph && !B->graph) {
      cudaGraph_t g = nullptr;
      const int64_t before = launch_count();
      BCK(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
      try {
        run_plan(B->plan_iter, B->cap_stream);
      } catch (...) {
        cudaStreamEndCapture(B->cap_stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      BCK(cudaStreamEndCapture(B->cap_stream, &g));
      B->graph_kernels = launch_count() - before;
      count_launch(-B->graph_kernels);
      BCK(cudaGraphInstantiate(&B->graph, g, 0));
      cudaGraphDestroy(g);
    }
    const int budget = o.maxit - total_it;
    int done_at = -1;
    auto check = [&](int k) -> bool {
      BCK(cudaEventSynchronize(B->ev[k & 1]));
      const int32_t* s4 = B->h_status + 4 * n * (1 + (k & 1));
      int32_t act = 0;
      for (int p = 0; p < n; ++p) {
        if (s4[4 * p + 1]) breakdown = true;
        act += s4[4 * p];
      }
      if (breakdown || act == 0) {
        done_at = k + 1;
        return true;
      }
      return false;
    };
    int it = 0;
    for (it = 0; it < budget; ++it) {
      if (B->graph && o.use_graph) {
        BCK(cudaGraphLaunch(B->graph, st));
        count_launch(B->graph_kernels);
      } else {
        run_plan(B->plan_iter, st);
      }
      BCK(cudaMemcpyAsync(B->h_status + 4 * n * (1 + (it & 1)), B->status_in, sizeof(int32_t) * 4 * n,
                          cudaMemcpyDeviceToHost, st));
      BCK(cudaEventRecord(B->ev[it & 1], st));
      if (it >= 1 && check(it - 1)) break;
    }
    if (done_at < 0 && it > 0 && !check(it - 1)) done_at = budget;
    BCK(cudaStreamSynchronize(st));
    total_it += done_at < 0 ? budget : done_at;
    for (int p = 0; p < n; ++p) {
      launch_add_to_f64(VEC_F32, ctx[p].D->n_b * B->C[p], ctx[p].D->xh, ctx[p].D->w32.x, st);
      check_launch();
    }
    if (breakdown) break;
  }
  for (int p = 0; p < n; ++p) {
    Device* D = ctx[p].D;
    launch_transform_bwd(D->xh, VEC_F64, B->nrhs[p], D->perm, D->n_b, D->s, x_dev[p], B->probs[p]->n, st);
    check_launch();
  }
  if (breakdown) {
    BCK(cudaStreamSynchronize(st));
    fail(AMGSYM_ERR_BREAKDOWN, "PCG breakdown in the batched solve");
  }
  const bool converged = active_out == 0;
  if (infos) {
    BCK(cudaStreamSynchronize(st));
    int64_t off = 0;
    for (int p = 0; p < n; ++p) {
      infos[p].iters = total_it;
      infos[p].outer_iters = outer;
      infos[p].converged = B->h_status[4 * p] == 0 ? 1 : 0;
      if (infos[p].relres) std::memcpy(infos[p].relres, B->h_relres + off, sizeof(double) * B->nrhs[p]);
      off += B->nrhs[p];
    }
  }
  return converged ? AMGSYM_OK : AMGSYM_NOT_CONVERGED;
}

}  // namespace amgsym

using namespace amgsym;

struct amgsym_batch {
  Batch* B = nullptr;
};

extern "C" amgsym_status amgsym_batch_create(const amgsym_t* problems, int32_t count, const int32_t* nrhs,
                                             amgsym_batch_t* out) {
  Batch* B = nullptr;
  try {
    if (!out) fail(AMGSYM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!problems || !nrhs || count < 1) fail(AMGSYM_ERR_ARG, "need at least one problem");
    B = new Batch();
    B->count = count;
    int nu = -1;
    for (int p = 0; p < count; ++p) {
      amgsym_t h = problems[p];
      Device* D = require_dev(h);
      if (p == 0) B->device_id = D->device_id;
      if (D->device_id != B->device_id) fail(AMGSYM_ERR_ARG, "all problems of a batch must be on one device");
      if (nrhs[p] < 1 || (int64_t)nrhs[p] * D->nb > 256) fail(AMGSYM_ERR_ARG, "nrhs * 2^s must be in [1, 256]");
      if (D->lv.size() < 2) fail(AMGSYM_ERR_STATE, "problem " + std::to_string(p) + " has a single-level hierarchy");
      if (D->singular) fail(AMGSYM_ERR_ARG, "problem " + std::to_string(p) + " is singular (pure Neumann): solve it alone");
      if (nu >= 0 && D->nu != nu) fail(AMGSYM_ERR_ARG, "all problems of a batch must use the same nu");
      nu = D->nu;
      B->probs.push_back(h);
      B->nrhs.push_back(nrhs[p]);
      B->C.push_back(nrhs[p] * D->nb);
    }
    BCK(cudaSetDevice(B->device_id));
    auto alloc = [&](size_t bytes) {
      void* q = nullptr;
      BCK(cudaMalloc(&q, bytes));
      B->owned.push_back(q);
      BCK(cudaMemset(q, 0, bytes));
      return q;
    };
    B->status_in = static_cast<int32_t*>(alloc(sizeof(int32_t) * 4 * count));
    B->status_out = static_cast<int32_t*>(alloc(sizeof(int32_t) * 4 * count));
    B->tol2_in = static_cast<double*>(alloc(sizeof(double) * count));
    B->tol2_out = static_cast<double*>(alloc(sizeof(double) * count));
    BCK(cudaMallocHost(&B->h_status, sizeof(int32_t) * 4 * count * 3));
    BCK(cudaMallocHost(&B->h_tol2, sizeof(double) * count));
    int64_t nr = 0;
    for (int p = 0; p < count; ++p) nr += nrhs[p];
    BCK(cudaMallocHost(&B->h_relres, sizeof(double) * nr));
    BCK(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    BCK(cudaStreamCreateWithFlags(&B->tune_stream, cudaStreamNonBlocking));
    BCK(cudaEventCreateWithFlags(&B->ev[0], cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&B->ev[1], cudaEventDisableTiming));
    auto* h = new amgsym_batch();
    h->B = B;
    *out = h;
    return AMGSYM_OK;
  } catch (const amgsym::Error& e) {
    batch_free(B);
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    batch_free(B);
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}

extern "C" amgsym_status amgsym_batch_solve(amgsym_batch_t b, const double* const* b_dev, double* const* x_dev,
                                            const amgsym_solve_opts* sopts, void* stream, amgsym_solve_info* infos) {
  try {
    if (!b || !b->B) fail(AMGSYM_ERR_ARG, "NULL batch");
    return batch_solve_impl(b->B, b_dev, x_dev, sopts, stream, infos);
  } catch (const amgsym::Error& e) {
    amgsym::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    amgsym::set_last_error("host allocation failed");
    return AMGSYM_ERR_OOM;
  }
}

extern "C" void amgsym_batch_destroy(amgsym_batch_t b) {
  if (!b) return;
  try {
    batch_free(b->B);
  } catch (...) {
  }
  delete b;
}
