"""OpenMP build of the oracle's conjugate gradients (ORACLE; test
infrastructure only, see ``oracle/__init__.py``).

``cg_omp.c`` is the iteration of ``oracle.solvers.cg`` written as plain C
loops so that the CPU baseline uses every host core.  ``build()`` compiles it
with the host C compiler into ``oracle/liboracle_cg.so`` (``__graft_entry__.build()``
calls it; ``cg`` also builds on first use).  It shares no code with the CUDA
library.
"""

from __future__ import annotations

import ctypes
import os
import platform
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cg_omp.c")
LIB = os.path.join(HERE, "liboracle_cg.so")
_lib = None


def build() -> str:
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no host C compiler for the oracle's OpenMP CG")
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle CG build failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.POINTER
        lib.oracle_cg.restype = ctypes.c_int
        lib.oracle_cg.argtypes = [ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_double),
                                  P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                  P(ctypes.c_int32)]
        _lib = lib
    return _lib


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cg(A, b, maxit: int, tol: float = 0.0, threads: int = 0):
    """CG from x = 0 on the CSR matrix A (scipy) for at most maxit
    iterations (tol = 0: exactly maxit).  Returns (x, info) with info =
    iters, seconds (loop wall time), threads, alphas, betas, relres (true)."""
    lib = _load()
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    v = np.ascontiguousarray(A.data, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n)
    al = np.zeros(max(maxit, 1))
    be = np.zeros(max(maxit, 1))
    sec = ctypes.c_double()
    nt = ctypes.c_int32()
    dp = ctypes.POINTER(ctypes.c_double)
    it = lib.oracle_cg(n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                       ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), v.ctypes.data_as(dp), b.ctypes.data_as(dp),
                       x.ctypes.data_as(dp), int(maxit), float(tol), int(threads), al.ctypes.data_as(dp),
                       be.ctypes.data_as(dp), ctypes.byref(sec), ctypes.byref(nt))
    if it < 0:
        raise MemoryError("oracle CG: allocation failed")
    rel = float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    return x, dict(iters=int(it), seconds=sec.value, threads=nt.value, alphas=al[:it], betas=be[:it], relres=rel)
