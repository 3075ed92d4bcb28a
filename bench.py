#!/usr/bin/env python3
"""Benchmark: symmetry-reduced AMG-PCG solves/s on the 256^3 stretched
variable-coefficient Poisson problem with three mirror symmetries.

One step = one solve (forward transform -> PCG / refinement -> backward
transform) of the RHS batch, setup excluded, inputs resident in HBM.
``value`` is the mixed-precision solve rate (FP32 inner PCG and V-cycle
inside FP64 iterative refinement, relative residual 1e-8); the FP64 solve of
the same problem is timed beside it.

Kernel measurement: ``amgsym_profile_step`` runs one solve step (transforms,
outer residual, PCG start, one PCG iteration) with CUDA events around every
launch on the solve's stream; ``kernels`` lists every kernel template with
its algorithmic bytes, time and fraction of the HBM copy peak, and
``roofline`` is the template with the largest share of a PCG iteration.
``vcycle`` sums the V-cycle's launches.  The reduced SpMM is also timed alone
with the L2 flushed (``reduced_spmm``).

Accuracy: ``accuracy`` gives the mixed-precision solution error of a uniform
256^3 problem (s = 3) against the oracle's exact sine-transform solve, per
right-hand side, and for the headline workload the bound kappa x relres with
kappa estimated by the oracle's CG-Lanczos run.  ``batched`` is the 64-problem
batched workload with the FP64 one-by-one solves of the same problems.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs N independent replicas (one problem is solved on one GPU: the
solve has no data-path exchange to shard), one per rank under
torch.distributed; rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import CONFIGS, batched_problem_specs, gaussian_logk, rhs_uniform  # noqa: E402

METRIC = "AMG-PCG solves/s + SpMM HBM GB/s, 256^3 s=3, mixed vs FP64 at rel-res 1e-8"
CFG = CONFIGS[3]
FIELD_SEED = 3000
CPU_SAMPLE_ITERS = 200

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel template in one solve step of this workload, from an ncu capture of
# the kernel sources whose SHA-256 is KERNEL_SOURCES_SHA256 (the committed
# profile summary gives the command).  Reported as roofline.traffic only while
# the sources are unchanged.
PROFILED_TRAFFIC = {
    "spmm_kernel<float,float,float,8,4,0,0,0>": 40902026,
    "spmm_kernel<float,float,float,8,1,0,0,1>": 161834445,
    "spmm_kernel<float,float,float,8,1,0,0,0>": 49454629,
    "spmm_kernel<float,float,float,8,1,1,0,1>": 275266304,
    "spmm_kernel<float,float,float,8,1,1,1,1>": 150906112,
    "spmm_kernel<float,float,float,4,4,0,0,0>": 9553536,
    "cg_update1_kernel<float>": 355761408,
    "cg_update2_kernel<float>": 152604928,
    "coarse_kernel<float>": 103424,
}
KERNEL_SOURCES = ("paper_2407_05930_gb300/csrc/k_spmm.cu", "paper_2407_05930_gb300/csrc/spmm_common.cuh",
                  "paper_2407_05930_gb300/csrc/k_misc.cu", "paper_2407_05930_gb300/csrc/dot.cuh",
                  "paper_2407_05930_gb300/csrc/stencil.cuh", "paper_2407_05930_gb300/csrc/coarse.cuh",
                  "paper_2407_05930_gb300/csrc/sell.cuh")
KERNEL_SOURCES_SHA256 = "63003fa80af8ea515d398f2376ba11e2580612e28b88acf4169daa0f18d74347"


def _kernel_sources_sha():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(sec: float, device=None) -> float:
    """The slowest rank's time (replicas: the job finishes with the last one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return sec
    t = torch.tensor([sec], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, sec_max: float, world: int) -> float:
    """Whole-job rate of `world` independent replicas: all units over the max time."""
    return world * units_per_rank / sec_max


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# CPU legs: the FP64 oracle (unpreconditioned CG on the full unreduced system,
# OpenMP over every host core)

def _oracle_operator():
    from oracle import fv, grid

    N, s = CFG["N"], CFG["s"]
    g = gaussian_logk(N, s, seed=FIELD_SEED, corr=8.0)
    A = fv.assemble(grid.widths(N, 1.5), np.exp(g))
    b = rhs_uniform(A.shape[0], 1, config=3)[0]
    return A, b


def _iters_to_tol(kappa: float):
    """Iterations of the oracle's CG to 1e-8 on this workload: the committed
    record of its full run when present, else the Chebyshev estimate
    ceil(sqrt(kappa)/2 ln(2/tol)) from the Lanczos kappa (a lower bound)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_cg_256cube.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("workload") == CFG["name"] and abs(rec.get("tol", 0) - CFG["tol"]) == 0:
            return int(rec["iters"]), "the oracle's full CG run to 1e-8 (tests/golden/oracle_cg_256cube.json)"
    except (OSError, ValueError, KeyError):
        pass
    it = int(np.ceil(0.5 * np.sqrt(kappa) * np.log(2.0 / CFG["tol"])))
    return it, f"ceil(sqrt(kappa)/2 ln(2/tol)) with the Lanczos kappa (a lower bound, so the rate is an upper bound)"


def _cpu_sample(A, b, iters: int):
    """Time `iters` iterations of the oracle's OpenMP CG on every host core."""
    from oracle import native, solvers

    cores = native.host_cores()
    _, info = native.cg(A, b, iters, 0.0, threads=cores)
    t_iter = info["seconds"] / max(1, info["iters"])
    kappa = solvers.lanczos_condition_estimate(info["alphas"], info["betas"])
    return t_iter, kappa, info["threads"], native.cpu_model()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    t0 = time.time()
    A, b = _oracle_operator()
    per_step = max(1, -(-CPU_SAMPLE_ITERS // max(1, args.steps)))
    from oracle import native

    native.cg(A, b, 2, 0.0, threads=native.host_cores())  # page in, spawn the threads
    for _ in range(args.warmup):
        native.cg(A, b, 1, 0.0, threads=native.host_cores())
    ts = []
    kappa = threads = model = None
    for _ in range(args.steps):
        t_iter, kappa, threads, model = _cpu_sample(A, b, per_step)
        ts.append(t_iter)
    t_iter = statistics.median(ts)
    it_needed, how = _iters_to_tol(kappa)
    if "golden" not in how:
        _, kappa, _, _ = _cpu_sample(A, b, CPU_SAMPLE_ITERS)  # a longer Lanczos run for the estimate
        it_needed, how = _iters_to_tol(kappa)
    solves_per_s = 1.0 / (t_iter * it_needed)
    sample = (f"{args.steps} steps x {per_step} CG iterations on the full {A.shape[0]}-unknown FP64 system, "
              f"OpenMP on {threads} cores ({model}); extrapolated to {it_needed} iterations to 1e-8 from {how}")
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": solves_per_s,
        "unit": "solves/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_iter * per_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": CFG["name"], "grid": "256^3", "s": 3, "nrhs": 1, "tol": CFG["tol"],
                   "solver": "oracle: unpreconditioned CG on the full unreduced FP64 system (oracle/cg_omp.c)"},
        "cpu_baseline": {"value": solves_per_s, "unit": "solves/s", "cores": threads, "cpu": model, "kind": "oracle",
                         "extrapolated": True, "sample": sample, "s_per_iter": t_iter},
        "e2e": {"value": solves_per_s, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.time() - t0,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


def _spmm_roofline(P, amg, torch, nrhs: int, reps: int = 30):
    """Time the reduced SpMM (FP32 values and vectors, interface fused) alone:
    per-launch CUDA events on the launching stream, L2 flushed between launches:
    a 256 MiB buffer is written (evicting every line) and then a second one is
    read, so the write-backs of the dirty flush lines happen before the timed
    launch instead of inside it."""
    sz = P.sizes()
    C = nrhs * P.nb
    n_b = P.n_b
    X = torch.randn((n_b, C), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clean = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sink = torch.empty((), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    ts = []
    for i in range(reps + 3):
        flush.zero_()
        torch.sum(clean, dim=0, out=sink)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        P.apply_reduced(X, Y, nrhs, amg.PREC_MIXED_FP32)
        e1.record(st)
        e1.synchronize()
        if i >= 3:
            ts.append(e0.elapsed_time(e1) * 1e-3)
    t = statistics.mean(ts)
    nnz = sz["nnz_inn"]
    words = (n_b + 31) // 32
    iface = words * 8 + (sz["n_iface_rows"] + 1) * 4 + sz["n_iface_rows"] * 4 + sz["n_iface_entries"] * (4 + 4 * P.nb)
    dia = P.level_dia(0, "A")
    if dia["ndiag"] > 0:
        # diagonal-offset form: the stored value arrays, no indices
        mat, storage = dia["nstored"] * n_b * 4, f"diagonal ({dia['ndiag']} diagonals, {dia['nstored']} stored)"
    else:
        mat, storage = nnz * (4 + 4) + 4 * (n_b + 1), "csr"
    algo = mat + C * 4 * (n_b + n_b) + iface
    return t, algo, storage


def _profile(P, b, x, nrhs, prec, reps=3, finest_hat=False):
    """Median over `reps` runs of amgsym_profile_step, launch by launch."""
    runs = [P.profile_step(b, x, nrhs, prec, finest_hat=finest_hat) for _ in range(reps)]
    recs = runs[0]
    for i, r in enumerate(recs):
        r["us"] = statistics.median(run[i]["us"] for run in runs if i < len(run))
    return recs


def _kernel_table(recs, peak):
    """Per kernel template: launches, bytes and time in one PCG iteration
    (phase 1) and in the once-per-step part (phase 0); the ncu DRAM bytes per
    launch of the committed capture while the kernel sources match it."""
    sha_ok = bool(KERNEL_SOURCES_SHA256) and _kernel_sources_sha() == KERNEL_SOURCES_SHA256
    groups = {}
    for r in recs:
        g = groups.setdefault((r["phase"], r["kernel"]), dict(kernel=r["kernel"], phase=r["phase"], launches=0,
                                                              bytes=0, us=0.0, roles=[]))
        g["launches"] += 1
        g["bytes"] += r["bytes"]
        g["us"] += r["us"]
        if r["role"] not in g["roles"]:
            g["roles"].append(r["role"])
    it_us = sum(g["us"] for g in groups.values() if g["phase"] == 1)
    out = []
    for g in sorted(groups.values(), key=lambda g: (-g["phase"], -g["us"])):
        gbs = g["bytes"] / (g["us"] * 1e-6) / 1e9 if g["us"] > 0 else 0.0
        e = dict(kernel=g["kernel"], per="iteration" if g["phase"] == 1 else "step", launches=g["launches"],
                 algo_bytes=g["bytes"], us=round(g["us"], 2), gbs=round(gbs, 1), frac=round(gbs / peak, 3),
                 roles="; ".join(g["roles"]))
        if g["phase"] == 1 and sha_ok and g["kernel"] in PROFILED_TRAFFIC:
            e["dram_bytes_per_launch"] = PROFILED_TRAFFIC[g["kernel"]]
        if g["phase"] == 1:
            e["share_of_iteration"] = round(g["us"] / it_us, 3)
        out.append(e)
    return out, it_us


def _uniform_accuracy(amg, torch, dev, nrhs=2):
    """Mixed-precision and FP64 solves of the uniform 256^3 problem (s = 3,
    k = 1) whose exact solution the oracle computes by sine transforms."""
    N, s = CFG["N"], CFG["s"]
    P = amg.Problem.structured(N, 0.0, None, s).setup()
    b_host = rhs_uniform(P.n, nrhs, config=30)
    b = torch.from_numpy(b_host).to(dev)
    xm, im = P.solve(b, tol=CFG["tol"], precision=amg.PREC_MIXED_FP32)
    xd, idd = P.solve(b, tol=CFG["tol"], precision=amg.PREC_FP64)
    out = dict(b=b_host, x_mixed=xm.cpu().numpy(), x_fp64=xd.cpu().numpy(), relres_mixed=im.relres.tolist(),
               relres_fp64=idd.relres.tolist())
    P.close()
    torch.cuda.empty_cache()
    return out


def _oracle_accuracy(u):
    """CPU leg: per-RHS solution error of the GPU solves against the oracle's
    exact DST solve, with the bound kappa x relres (kappa from the closed form)."""
    from oracle import solvers

    N = CFG["N"]
    xo = solvers.dst_solve(N, u["b"])
    # uniform cube: every axis has the same weight, so lambda_max / lambda_min
    # of the Kronecker sum is sin^2(N pi / 2N) / sin^2(pi / 2N)
    kappa = 1.0 / np.sin(np.pi / (2.0 * N[0])) ** 2
    err_m = [float(np.linalg.norm(u["x_mixed"][r] - xo[r]) / np.linalg.norm(xo[r])) for r in range(xo.shape[0])]
    err_d = [float(np.linalg.norm(u["x_fp64"][r] - xo[r]) / np.linalg.norm(xo[r])) for r in range(xo.shape[0])]
    return dict(workload="3d7pt_uniform_256cube_s3 (k = 1, no stretching), 2 uniform[-1,1] RHS, tol 1e-8",
                oracle="oracle.solvers.dst_solve (exact sine-transform solve)",
                err_mixed_per_rhs=err_m, err_fp64_per_rhs=err_d, relres_mixed=u["relres_mixed"],
                relres_fp64=u["relres_fp64"], kappa=kappa,
                bound_kappa_relres_mixed=[kappa * r for r in u["relres_mixed"]])


def run_batched(args, inline=False):
    """The batched workload: 64 problems, cube edge N uniform over the even
    integers in [32, 160], s uniform in {1, 2, 3}, 16 uniform[-1, 1] RHS each,
    mixed precision to 1e-8, one batched solve per step; beside it the FP64
    reduced solves of the same problems one by one (every problem, timed).
    inline: return the record instead of printing a JSON line."""
    import torch

    import paper_2407_05930_gb300 as amg

    dev = torch.device("cuda", torch.cuda.current_device())
    specs = batched_problem_specs(count=args.batch_count)
    t0 = time.time()
    probs, bs = [], []
    for k, sp in enumerate(specs):
        P = amg.Problem.structured(sp["N"], 0.0, None, sp["s"]).setup(coarse_max=64)
        probs.append(P)
        bs.append(torch.from_numpy(rhs_uniform(P.n, 16, config=4000 + k)).to(dev))
    t_setup = time.time() - t0
    B = amg.Batch(probs, [16] * len(probs))
    kw = dict(tol=1e-8, precision=amg.PREC_MIXED_FP32, tune=0 if args.no_tune else 1)
    xs = [torch.empty_like(b) for b in bs]
    steps = args.batch_steps if inline else args.steps
    warm = 1 if inline else args.warmup
    for _ in range(max(1, warm)):
        _, res = B.solve(bs, xs, **kw)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = amg.kernel_launches()
    torch.cuda.nvtx.range_push("timed_batched")
    e0.record(st)
    for _ in range(steps):
        _, res = B.solve(bs, xs, **kw)
    e1.record(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    launches = amg.kernel_launches() - l0
    nsolves = 16 * len(probs)
    # FP64 reduced solves of the same problems, one at a time, every problem:
    # one untimed solve each (work arrays, graph capture), then one timed
    for i in range(len(probs)):
        probs[i].solve(bs[i], xs[i], tol=1e-8, precision=amg.PREC_FP64)
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(len(probs)):
        probs[i].solve_async(bs[i], xs[i], 16, tol=1e-8, precision=amg.PREC_FP64)
    e1.record(st)
    torch.cuda.synchronize()
    sec64 = e0.elapsed_time(e1) * 1e-3
    rec = {
        "value": nsolves * steps / sec, "unit": "solves/s", "steps": steps, "ms_per_step": sec / steps * 1e3,
        "workload": CONFIGS[4]["name"], "problems": len(probs), "cells": int(sum(p.n for p in probs)),
        "rhs_per_problem": 16, "tol": 1e-8, "precision": "FP32 V-cycle + FP64 refinement",
        "tiles": "fixed from row lengths" if args.no_tune else "autotuned per problem and matrix",
        "inner_iters": res[0].iters, "outer_iters": res[0].outer_iters,
        "max_relres": float(max(np.max(r.relres) for r in res)), "all_converged": all(r.converged for r in res),
        "fp64_sequential": {"value": nsolves / sec64, "unit": "solves/s", "ms": sec64 * 1e3,
                            "sample": f"all {len(probs)} problems, 16 RHS each, solved one by one in FP64 "
                                      "(reduced AMG-PCG to 1e-8), one timed pass after one untimed pass"},
        "gpu_launches": int(launches), "setup_s": round(t_setup, 1),
    }
    del B
    for P in probs:
        P.close()
    torch.cuda.empty_cache()
    if inline:
        return rec
    line = {"metric": "batched AMG-PCG solves/s (64 problems x 16 RHS, mixed precision, rel-res 1e-8)",
            "value": rec["value"], "unit": "solves/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": rec["workload"], "problems": rec["problems"], "cells": rec["cells"],
                       "rhs_per_problem": 16, "sizes": [sp["N"][0] for sp in specs], "s": [sp["s"] for sp in specs]},
            **{k: rec[k] for k in ("tiles", "inner_iters", "outer_iters", "max_relres", "all_converged",
                                   "fp64_sequential", "gpu_launches", "setup_s")}}
    print(json.dumps(line), flush=True)


def run_model_tables(args):
    """The paper's model problem (Sec. 2.2, eq. "modelproblem": Neumann on
    every wall, 64^3 cells, tanh stretching 1.5, random compatible f):
    iteration counts of this library's solvers next to the paper's Tables
    "lrcamg" (GMRES + LRCAMG(k)) and "amgr" (PCG + AMGR), to relative
    residual 1e-8.  PCG with I (x) M_inn^{-1} (s = 0: AMG of the full
    domain), PCG with AMGR, GMRES(60) with LRCAMG(k) and PCG with LRCFSAI(k),
    k = 0, 1, 2, 4, 8, 16 (Table "lrcfsai")."""
    import torch

    import paper_2407_05930_gb300 as amg
    from oracle import fv, grid

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N = (args.model_grid,) * 3
    h = grid.widths(N, 1.5)
    ks = (0, 1, 2, 4, 8, 16)
    pcg, gm, amgr, fs, relmax = {}, {}, {}, {}, 0.0
    gm_setup, fs_setup = {}, {}
    for s in range(4):
        P = amg.Problem.structured(N, 1.5, None, s, bc="neumann").setup(amgr=1)
        f = np.random.default_rng(94).uniform(-1.0, 1.0, P.n)
        b = f * fv.cell_volumes(h)
        b -= b.mean()
        bt = torch.from_numpy(b).to(dev)
        x, info = P.solve(bt, tol=1e-8)
        pcg[s] = info.iters
        relmax = max(relmax, float(np.max(info.relres)))
        x, info = P.solve(bt, tol=1e-8, preconditioner=amg.PC_AMGR)
        amgr[s] = info.iters
        relmax = max(relmax, float(np.max(info.relres)))
        row, srow = [], []
        for k in ks:
            t0 = time.perf_counter()
            P.lrc_setup(k)
            srow.append(round(time.perf_counter() - t0, 3))
            x, info = P.solve_gmres(bt, restart=60, lrc=k > 0, tol=1e-8, maxit=400)
            row.append(info.iters if info.converged else None)
            relmax = max(relmax, float(np.max(info.relres)))
        gm[s], gm_setup[s] = row, srow
        row, srow = [], []
        for k in ks:
            t0 = time.perf_counter()
            if k:
                P.lrcfsai_setup(k)
            srow.append(round(time.perf_counter() - t0, 3))
            x, info = P.solve_fsai(bt, lrc=k > 0, tol=1e-8, maxit=5000)
            row.append(info.iters if info.converged else None)
            relmax = max(relmax, float(np.max(info.relres)))
        fs[s], fs_setup[s] = row, srow
        P.close()
    line = {"workload": f"neumann model problem {N[0]}^3, tanh 1.5, s = 0..3, relres 1e-8",
            "pcg_I_x_Minn": pcg, "pcg_amgr": amgr, "gmres_lrcamg": {"k": list(ks), "iters_by_s": gm, "setup_s_by_s": gm_setup},
            "pcg_lrcfsai": {"k": list(ks), "iters_by_s": fs, "setup_s_by_s": fs_setup},
            "max_relres": relmax,
            "paper_64cube": {"gmres_AMG": [6, 6, 6, 6], "gmres_LRCAMG": {"0": [6, 23, 29, 29], "1": [9, 23, 26, 24],
                             "2": [9, 23, 22, 24], "4": [9, 19, 21, 20], "8": [9, 17, 18, 18],
                             "16": [9, 15, 16, 15]}, "pcg_AMGR": [6, 9, 9, 9],
                             "pcg_LRCFSAI": {"FSAI": [291, 220, 173, 121], "0": [291, 241, 193, 149],
                                             "1": [228, 194, 146, 106], "2": [228, 172, 124, 92],
                                             "4": [186, 136, 107, 83], "8": [131, 111, 81, 61],
                                             "16": [113, 82, 63, 50]}}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch

    import paper_2407_05930_gb300 as amg

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    N, s, nrhs, tol = CFG["N"], CFG["s"], args.nrhs, CFG["tol"]

    if args.profile_only and args.profile_grid != N[0]:
        N = (args.profile_grid,) * 3  # a smaller case of the same workload, for ncu pass counts
    t_setup = time.time()
    g = gaussian_logk(N, s, seed=FIELD_SEED, corr=8.0)
    # amgr=1 also builds AMGR (Sec. 3.2) beside the I (x) M_inn hierarchy, for its variant line
    with_amgr = not args.profile_only or args.profile_only.startswith("amgr")
    extra = {}
    for kv in args.setup_opt:  # --profile-only captures of the optional kernel forms
        key, _, val = kv.partition("=")
        extra[key] = type(getattr(amg.default_opts(), key))(val)
    P = amg.Problem.structured(N, 1.5, g, s).setup(precisions=3, amgr=1 if with_amgr else 0, **extra)
    b_host = rhs_uniform(P.n, nrhs, config=3)
    b = torch.from_numpy(b_host).to(dev)
    x = torch.empty_like(b)
    t_setup = time.time() - t_setup

    mixed = dict(tol=tol, precision=amg.PREC_MIXED_FP32)
    fp64 = dict(tol=tol, precision=amg.PREC_FP64)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    if args.profile_only:
        # one warm-up solve, then the marked work only (for ncu launch lists)
        kw = fp64 if args.profile_only == "fp64" else mixed
        if args.profile_only.startswith("amgr"):
            kw = dict(mixed, preconditioner=amg.PC_AMGR)
        P.solve(b, x, **kw)
        torch.cuda.synchronize()
        if args.profile_only in ("step", "amgr_step"):
            pc = amg.PC_AMGR if args.profile_only == "amgr_step" else amg.PC_AMG
            torch.cuda.nvtx.range_push("profile_step")
            recs = P.profile_step(b, x, nrhs, amg.PREC_MIXED_FP32, preconditioner=pc)
            torch.cuda.nvtx.range_pop()
            for r in recs:
                print(json.dumps(r))
            return
        torch.cuda.nvtx.range_push("timed_" + args.profile_only)
        P.solve_async(b, x, nrhs, **kw)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        torch.cuda.nvtx.range_push("roofline")
        t_k, algo, _ = _spmm_roofline(P, amg, torch, nrhs, reps=3)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_only": args.profile_only, "spmm_us": t_k * 1e6}))
        return

    # warm-up (also captures the CUDA graphs)
    for _ in range(args.warmup):
        _, info_m = P.solve(b, x, **mixed)
    for _ in range(max(1, args.warmup)):
        _, info_d = P.solve(b, x, **fp64)
    torch.cuda.synchronize()

    def timed(kw, steps):
        barrier()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = amg.kernel_launches()
        e0.record(st)
        for _ in range(steps):
            P.solve_async(b, x, nrhs, **kw)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
        sec = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dev)
        return sec, amg.kernel_launches() - l0

    nvtx = torch.cuda.nvtx
    with ClockSampler(torch.cuda.current_device()) as clk:
        nvtx.range_push("timed_mixed")
        sec_m, launches_m = timed(mixed, args.steps)
        nvtx.range_pop()
    clocks = clk.summary()
    nvtx.range_push("timed_fp64")
    steps_d = max(1, args.steps // 2)
    sec_d, launches_d = timed(fp64, steps_d)
    nvtx.range_pop()

    # end to end through the public API: pinned host b -> device -> solve -> host x
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        b.copy_(b_pin, non_blocking=True)
        P.solve_async(b, x, nrhs, **mixed)
        x_pin.copy_(x, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    sec_e = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dev)

    # variant: finest-level V-cycle residuals with the interface-corrected
    # blocks A^_i instead of A_inn (same hierarchy)
    hat = dict(mixed, finest_hat=1)
    P.solve(b, x, **hat)
    sec_h, _ = timed(hat, steps_d)
    _, info_h = P.solve(b, x, **hat)

    # variant: AMGR (Sec. 3.2, the paper's multigrid reduction) as the PCG
    # preconditioner of the same problem, mixed and FP64
    amgr_m = dict(mixed, preconditioner=amg.PC_AMGR)
    amgr_d = dict(fp64, preconditioner=amg.PC_AMGR)
    P.solve(b, x, **amgr_m)
    sec_am, _ = timed(amgr_m, steps_d)
    _, info_am = P.solve(b, x, **amgr_m)
    P.solve(b, x, **amgr_d)
    sec_ad, _ = timed(amgr_d, steps_d)
    _, info_ad = P.solve(b, x, **amgr_d)

    # the solver's own true residuals of the timed solves
    _, info_m = P.solve(b, x, **mixed)
    _, info_d = P.solve(b, x, **fp64)

    peak, peak_kind = _peaks()
    # per-launch timing of one solve step (mixed precision)
    nvtx.range_push("profile_step")
    recs = _profile(P, b, torch.empty_like(b), nrhs, amg.PREC_MIXED_FP32)
    nvtx.range_pop()
    kernels, it_us = _kernel_table(recs, peak)
    it_kernels = [k for k in kernels if k["per"] == "iteration"]
    dom = max(it_kernels, key=lambda k: k["us"])
    vrec = [r for r in recs if r["phase"] == 1 and r["level"] >= 0]
    v_bytes = sum(r["bytes"] for r in vrec)
    v_us = sum(r["us"] for r in vrec)
    # the whole V-cycle as one call (launch gaps included), events on the stream
    C = nrhs * P.nb
    R = torch.randn((P.n_b, C), dtype=torch.float32, device=dev)
    Z = torch.empty_like(R)
    for _ in range(3):
        P.vcycle(R, Z, nrhs, amg.PREC_MIXED_FP32)
    e0.record(st)
    for _ in range(10):
        P.vcycle(R, Z, nrhs, amg.PREC_MIXED_FP32)
    e1.record(st)
    torch.cuda.synchronize()
    v_call_us = e0.elapsed_time(e1) * 1e3 / 10
    del R, Z

    # the AMGR variant's iteration, launch by launch: its heaviest kernel templates
    recs_a = [P.profile_step(b, torch.empty_like(b), nrhs, amg.PREC_MIXED_FP32, preconditioner=amg.PC_AMGR)
              for _ in range(3)]
    agg_a = {}
    for i, r in enumerate(recs_a[0]):
        if r["phase"] != 1:
            continue
        us = statistics.median(run[i]["us"] for run in recs_a if i < len(run))
        e = agg_a.setdefault(r["kernel"], {"kernel": r["kernel"], "launches": 0, "us": 0.0, "bytes": 0})
        e["launches"] += 1
        e["us"] += us
        e["bytes"] += r["bytes"]
    it_a = sum(e["us"] for e in agg_a.values())
    amgr_kernels = []
    for e in sorted(agg_a.values(), key=lambda e: -e["us"])[:6]:
        gbs = e["bytes"] / (e["us"] * 1e-6) / 1e9
        amgr_kernels.append({"kernel": e["kernel"], "launches": e["launches"], "us": round(e["us"], 1),
                             "share_of_iteration": round(e["us"] / it_a, 3), "algo_GBps": round(gbs),
                             "frac": round(gbs / peak, 3)})

    nvtx.range_push("roofline")
    t_k, algo, storage = _spmm_roofline(P, amg, torch, nrhs)
    nvtx.range_pop()
    achieved_k = algo / t_k / 1e9

    sha_ok = KERNEL_SOURCES_SHA256 and _kernel_sources_sha() == KERNEL_SOURCES_SHA256
    dom_gbs = dom["algo_bytes"] / (dom["us"] * 1e-6) / 1e9
    traffic = PROFILED_TRAFFIC.get(dom["kernel"]) if sha_ok else None
    value = replica_rate(nrhs * args.steps, sec_m, ws)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sec_m / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {
            "workload": CFG["name"], "grid": "256^3 cells, tanh stretching 1.5", "s": s, "nrhs": nrhs,
            "tol": tol, "k": "exp(g), g mirror-symmetric smoothed Gaussian (corr 8 cells, sigma 1)",
            "precision": "FP32 inner PCG + FP32 V-cycle inside FP64 iterative refinement",
            "l2": "working set (~2 GB of matrices and vectors per solve) larger than L2",
            "parallelism": "replicas" if ws > 1 else "single GPU",
        },
        "iters": {"mixed_inner": info_m.iters, "mixed_outer": info_m.outer_iters, "fp64": info_d.iters,
                  "relres_mixed": float(np.max(info_m.relres)), "relres_fp64": float(np.max(info_d.relres))},
        "fp64": {"value": ws * nrhs * steps_d / sec_d, "unit": "solves/s", "ms_per_step": sec_d / steps_d * 1e3},
        "variant_finest_hat": {"value": ws * nrhs * steps_d / sec_h, "unit": "solves/s",
                               "inner_iters": info_h.iters, "outer_iters": info_h.outer_iters,
                               "relres": float(np.max(info_h.relres))},
        "variant_amgr": {"value": ws * nrhs * steps_d / sec_am, "unit": "solves/s",
                         "inner_iters": info_am.iters, "outer_iters": info_am.outer_iters,
                         "relres": float(np.max(info_am.relres)),
                         "fp64": {"value": ws * nrhs * steps_d / sec_ad, "unit": "solves/s",
                                  "iters": info_ad.iters, "relres": float(np.max(info_ad.relres))},
                         "preconditioner": "AMGR V(1,1): populated coarsening MIS(T^1) + interface, "
                                           "P = I (x) [W; I] extended+i, block-FSAI top smoother, "
                                           "standard AMG of A_c = P^T A P (its level-0 products in "
                                           "the transformed basis)",
                         "iteration_us_kernels": round(it_a, 1), "kernels": amgr_kernels},
        "e2e": {"value": ws * nrhs * args.steps / sec_e, "unit": "solves/s",
                "h2d_bytes_per_step": int(b_pin.numel() * 8), "d2h_bytes_per_step": int(x_pin.numel() * 8)},
        "roofline": {"bound": "hbm", "kernel": dom["kernel"], "roles": dom["roles"],
                     "share_of_iteration": dom["share_of_iteration"], "launches_per_iteration": dom["launches"],
                     "achieved": dom_gbs, "peak": peak, "unit": "GB/s", "frac": dom_gbs / peak,
                     "peak_kind": peak_kind, "algo_bytes_per_launch": dom["algo_bytes"] / dom["launches"],
                     "launch_us": dom["us"] / dom["launches"], "traffic": traffic,
                     "timing": "CUDA events around each launch of one solve step on the solve's stream "
                               "(amgsym_profile_step), median of 3"},
        "kernels": kernels,
        "iteration": {"us_kernels": round(it_us, 1),
                      "us_measured": round(sec_m / args.steps * 1e6 / max(1, info_m.iters), 1),
                      "algo_bytes": sum(r["bytes"] for r in recs if r["phase"] == 1)},
        "vcycle": {"algo_bytes": v_bytes, "us_kernels": round(v_us, 1), "gbs": v_bytes / (v_us * 1e-6) / 1e9,
                   "frac": v_bytes / (v_us * 1e-6) / 1e9 / peak, "launches": len(vrec),
                   "us_call": round(v_call_us, 1)},
        "reduced_spmm": {"kernel": "spmm_kernel<float,float,float,8,1,1,1,1> alone (no dot: 8,1,0,1,1), L2 flushed",
                         "storage": storage, "algo_bytes_per_launch": algo, "launch_us": t_k * 1e6,
                         "achieved": achieved_k, "frac": achieved_k / peak},
        "gpu_launches": int(launches_m),
        "clocks": clocks,
        "setup_s": t_setup,
    }
    del P
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_accuracy:
        line["accuracy"] = {"uniform": _uniform_accuracy(amg, torch, dev)}
    if rank == 0 and ws == 1 and not args.no_batched:
        line["batched"] = run_batched(args, inline=True)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # CPU leg: the oracle on every host core, and the oracle's references
        A, bo = _oracle_operator()
        t_iter, kappa, threads, model = _cpu_sample(A, bo, CPU_SAMPLE_ITERS)
        del A
        it_needed, how = _iters_to_tol(kappa)
        line["cpu_baseline"] = {
            "value": 1.0 / (t_iter * it_needed), "unit": "solves/s", "cores": threads, "cpu": model,
            "kind": "oracle", "extrapolated": True, "s_per_iter": t_iter,
            "sample": f"{CPU_SAMPLE_ITERS} iterations of the oracle's unpreconditioned FP64 CG on the full "
                      f"{P_n(N)}-unknown system, OpenMP on {threads} cores ({model}); extrapolated to "
                      f"{it_needed} iterations to 1e-8 from {how}",
        }
        if "accuracy" in line:
            u = line["accuracy"].pop("uniform")
            line["accuracy"]["uniform"] = _oracle_accuracy(u)
        line.setdefault("accuracy", {})["headline"] = {
            "relres_mixed": line["iters"]["relres_mixed"], "kappa_lanczos": kappa,
            "bound_kappa_relres": kappa * line["iters"]["relres_mixed"],
            "note": "||x - x*||/||x*|| <= kappa(A) relres; kappa from the Ritz values of the oracle's "
                    f"{CPU_SAMPLE_ITERS}-iteration CG-Lanczos run (an estimate from below)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def P_n(N):
    return int(np.prod(N))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the uniform 256^3 accuracy solve")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload sub-object")
    ap.add_argument("--batch-steps", type=int, default=2, help="timed batched solves in the default line")
    ap.add_argument("--workload", choices=["256cube", "batched", "model"], default="256cube")
    ap.add_argument("--model-grid", type=int, default=64, help="model-problem tables: cells per axis")
    ap.add_argument("--profile-grid", type=int, default=256, help="--profile-only: cells per axis")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-tune", action="store_true", help="batched: fixed tiles instead of the autotuner")
    ap.add_argument("--setup-opt", action="append", default=[], metavar="KEY=VALUE",
                    help="--profile-only: an amgsym_opts field for the setup (e.g. sell=1)")
    ap.add_argument("--profile-only", choices=["mixed", "fp64", "step", "amgr", "amgr_step"], default=None,
                    help="run one marked solve (or one profiled step) and nothing else (for ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "model":
        run_model_tables(args)
    elif args.workload == "batched":
        import torch

        torch.cuda.set_device(0)
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
