#!/usr/bin/env python3
"""Benchmark: symmetry-reduced AMG-PCG solves/s on the 256^3 stretched
variable-coefficient Poisson problem with three mirror symmetries.

One step = one solve (forward transform -> PCG / refinement -> backward
transform) of the RHS batch, setup excluded, inputs resident in HBM.
``value`` is the mixed-precision solve rate (FP32 inner PCG and V-cycle
inside FP64 iterative refinement, relative residual 1e-8); the FP64 solve of
the same problem is timed beside it.  The dominant kernel (the reduced SpMM,
FP32 values and vectors) is timed on its own for the roofline entry.

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

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the reduced SpMM on this workload, from an ncu capture of the kernel sources
# with this SHA-256 (profiles/spmm_reduced_fp32_256cube_s3.md).  Reported as
# roofline.traffic only while the sources are unchanged.
SPMM_TRAFFIC_BYTES = 152.2e6
SPMM_SOURCES = ("paper_2407_05930_gb300/csrc/k_spmm.cu", "paper_2407_05930_gb300/csrc/spmm_common.cuh")
SPMM_SOURCES_SHA256 = "6f21e8049d657ebfb1561ca16bfa1536f1a631888c803285fb6fa1b1ed3086a2"


def _spmm_sources_sha():
    import hashlib

    h = hashlib.sha256()
    for f in SPMM_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()
CFG = CONFIGS[3]
FIELD_SEED = 3000


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
# Reference arm: the FP64 CPU oracle (unpreconditioned CG on the full system)

def _oracle_sample(steps: int, warmup: int, iters_per_step: int):
    from oracle import fv, grid, solvers

    N, s = CFG["N"], CFG["s"]
    g = gaussian_logk(N, s, seed=FIELD_SEED, corr=8.0)
    h = grid.widths(N, 1.5)
    A = fv.assemble(h, np.exp(g))
    b = rhs_uniform(A.shape[0], 1, config=3)[0]
    al_all, be_all = [], []
    times = []
    for k in range(warmup + steps):
        t, al, be = solvers.cg_sample(A, b, iters_per_step if k >= warmup else 1)
        if k >= warmup:
            times.append(t)
    # Lanczos estimate from one contiguous run of the CG recurrence
    t, al, be = solvers.cg_sample(A, b, max(iters_per_step * 4, 40))
    kappa = solvers.lanczos_condition_estimate(al, be)
    t_iter = statistics.median(times)
    it_est = int(np.ceil(0.5 * np.sqrt(kappa) * np.log(2.0 / CFG["tol"])))
    return t_iter, kappa, it_est, A.shape[0]


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    t0 = time.time()
    t_iter, kappa, it_est, n = _oracle_sample(args.steps, args.warmup, 5)
    solves_per_s = 1.0 / (t_iter * it_est)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": solves_per_s,
        "unit": "solves/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_iter * 5 * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": CFG["name"], "grid": "256^3", "s": 3, "nrhs": 1, "tol": CFG["tol"],
                   "solver": "oracle: unpreconditioned CG on the full unreduced FP64 system (scipy CSR)"},
        "cpu_baseline": {
            "value": solves_per_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{args.steps} steps x 5 CG iterations on the full {n}-unknown system; "
                      f"iterations to 1e-8 extrapolated as ceil(sqrt(kappa)/2 ln(2/tol)) = {it_est} "
                      f"with kappa >= {kappa:.3g} from the CG-Lanczos Ritz values (an underestimate, "
                      "so this rate is an upper bound)",
        },
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
    iface = words * 8 + (sz["n_iface_rows"] + 1) * 4 + sz["n_iface_entries"] * (4 + 4 * P.nb)
    dia = P.level_dia(0, "A")
    if dia["ndiag"] > 0:
        # diagonal-offset form: the stored value arrays, no indices
        mat, storage = dia["nstored"] * n_b * 4, f"diagonal ({dia['ndiag']} diagonals, {dia['nstored']} stored)"
    else:
        mat, storage = nnz * (4 + 4) + 4 * (n_b + 1), "csr"
    algo = mat + C * 4 * (n_b + n_b) + iface
    return t, algo, storage


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

    t_setup = time.time()
    g = gaussian_logk(N, s, seed=FIELD_SEED, corr=8.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(precisions=3)
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
        # one warm-up and one NVTX-marked solve of the requested arithmetic, for
        # ncu launch lists (no other work in the process)
        kw = mixed if args.profile_only == "mixed" else fp64
        P.solve(b, x, **kw)
        torch.cuda.synchronize()
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
    sec_d, launches_d = timed(fp64, max(1, args.steps // 2))
    nvtx.range_pop()
    steps_d = max(1, args.steps // 2)

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
    sec_h, _ = timed(hat, max(1, args.steps // 2))
    _, info_h = P.solve(b, x, **hat)

    # accuracy of the timed solves against the oracle's residual definition is
    # covered by the tests; here report the solver's own true residuals
    _, info_m = P.solve(b, x, **mixed)
    _, info_d = P.solve(b, x, **fp64)

    nvtx.range_push("roofline")
    t_k, algo, storage = _spmm_roofline(P, amg, torch, nrhs)
    nvtx.range_pop()
    peak, peak_kind = _peaks()
    achieved = algo / t_k / 1e9

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
        "variant_finest_hat": {"value": ws * nrhs * max(1, args.steps // 2) / sec_h, "unit": "solves/s",
                               "inner_iters": info_h.iters, "outer_iters": info_h.outer_iters,
                               "relres": float(np.max(info_h.relres))},
        "e2e": {"value": ws * nrhs * args.steps / sec_e, "unit": "solves/s",
                "h2d_bytes_per_step": int(b_pin.numel() * 8), "d2h_bytes_per_step": int(x_pin.numel() * 8)},
        "roofline": {"bound": "hbm", "kernel": "spmm_kernel<float,float,float> (reduced SpMM, interface fused)",
                     "storage": storage,
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "algo_bytes_per_launch": algo, "launch_us": t_k * 1e6,
                     "traffic": SPMM_TRAFFIC_BYTES if _spmm_sources_sha() == SPMM_SOURCES_SHA256 else None},
        "gpu_launches": int(launches_m),
        "clocks": clocks,
        "setup_s": t_setup,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t_iter, kappa, it_est, n = _oracle_sample(1, 0, 5)
        line["cpu_baseline"] = {
            "value": 1.0 / (t_iter * it_est), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"5 iterations of the oracle's unpreconditioned FP64 CG on the full {n}-unknown system; "
                      f"iterations to 1e-8 extrapolated as ceil(sqrt(kappa)/2 ln(2/tol)) = {it_est}, "
                      f"kappa >= {kappa:.3g} from CG-Lanczos Ritz values (so an upper bound on the rate)",
        }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batched(args):
    """The batched workload: 64 problems, cube edge N uniform over the even
    integers in [32, 160], s uniform in {1, 2, 3}, 16 uniform[-1, 1] RHS each,
    mixed precision to 1e-8, one batched solve per step.  Prints its own JSON
    line (the default line is the 256^3 workload)."""
    import torch

    import paper_2407_05930_gb300 as amg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
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
    for _ in range(args.warmup):
        _, res = B.solve(bs, xs, **kw)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = amg.kernel_launches()
    torch.cuda.nvtx.range_push("timed_batched")
    e0.record(st)
    for _ in range(args.steps):
        _, res = B.solve(bs, xs, **kw)
    e1.record(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    launches = amg.kernel_launches() - l0
    nsolves = 16 * len(probs)
    # FP64 reduced solves of the same problems one at a time (a sample of
    # `fp64_sample` problems, rate extrapolated by unknowns x RHS)
    samp = list(range(0, len(probs), max(1, len(probs) // args.fp64_sample)))[: args.fp64_sample]
    work_all = sum(p.n for p in probs)
    work_s = sum(probs[i].n for i in samp)
    for i in samp:
        probs[i].solve(bs[i], tol=1e-8, precision=amg.PREC_FP64)
    torch.cuda.synchronize()
    e0.record(st)
    for i in samp:
        probs[i].solve(bs[i], tol=1e-8, precision=amg.PREC_FP64)
    e1.record(st)
    torch.cuda.synchronize()
    sec64 = e0.elapsed_time(e1) * 1e-3 * work_all / work_s
    line = {
        "metric": "batched AMG-PCG solves/s (64 problems x 16 RHS, mixed precision, rel-res 1e-8)",
        "value": nsolves * args.steps / sec, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": CONFIGS[4]["name"], "problems": len(probs),
                   "cells": int(sum(p.n for p in probs)), "rhs_per_problem": 16,
                   "sizes": [sp["N"][0] for sp in specs], "s": [sp["s"] for sp in specs]},
        "tiles": "fixed from row lengths" if args.no_tune else "autotuned per problem and matrix",
        "inner_iters": res[0].iters, "outer_iters": res[0].outer_iters,
        "max_relres": float(max(np.max(r.relres) for r in res)), "all_converged": all(r.converged for r in res),
        "fp64_sequential": {"value": nsolves / sec64, "unit": "solves/s",
                            "sample": f"{len(samp)} of {len(probs)} problems solved one by one in FP64, "
                                      "time scaled by unknowns"},
        "gpu_launches": int(launches), "setup_s": t_setup,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["256cube", "batched"], default="256cube")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--no-tune", action="store_true", help="batched: fixed tiles instead of the autotuner")
    ap.add_argument("--fp64-sample", type=int, default=8)
    ap.add_argument("--profile-only", choices=["mixed", "fp64"], default=None,
                    help="run one marked solve and the roofline SpMM only (for ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
