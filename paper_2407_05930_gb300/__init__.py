"""Python binding of the amgsym C ABI (``include/amgsym.h``).

Symmetry-reduced AMG-preconditioned CG for the discrete Poisson equation
(arXiv 2407.05930, Alg. 1 with the preconditioner ``I (x) M_inn^{-1}``).
This module only marshals arguments: every step of the solve runs in the
CUDA kernels of ``libamgsym.so``.  PyTorch supplies device memory and the
current stream.  There is no CPU fallback: importing fails if the library
has not been built (``paper_2407_05930_gb300.build.build()``), and the device
entry points fail if no CUDA device is present.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamgsym.so")

PREC_FP64 = 0
PREC_MIXED_FP32 = 1
PREC_MIXED_BF16 = 2

BC = {"dirichlet": 0, "neumann": 1}

PC_AMG = 0
PC_AMGR = 1

STATUS = {
    0: "OK",
    1: "NOT_CONVERGED",
    -1: "ERR_ARG",
    -2: "ERR_MAP",
    -3: "ERR_NOT_SYMMETRIC",
    -4: "ERR_NOT_SPD",
    -5: "ERR_BREAKDOWN",
    -6: "ERR_CUDA",
    -7: "ERR_OOM",
    -8: "ERR_DEVICE_TIMEOUT",
    -9: "ERR_STATE",
}


class AmgsymError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Opts(ctypes.Structure):
    _fields_ = [
        ("strength_theta", ctypes.c_double),
        ("interp_trunc", ctypes.c_double),
        ("interp_max_elems", ctypes.c_int32),
        ("max_levels", ctypes.c_int32),
        ("coarse_max", ctypes.c_int32),
        ("fsai_max_lower", ctypes.c_int32),
        ("omega_scale", ctypes.c_double),
        ("nu", ctypes.c_int32),
        ("precisions", ctypes.c_int32),
        ("host_only", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("coarse_drop", ctypes.c_double),
        ("dia_max_diag", ctypes.c_int32),
        ("fuse_rows", ctypes.c_int32),
        ("fsai_max_lower_coarse", ctypes.c_int32),
        ("halo_kb", ctypes.c_int32),
        ("amgr", ctypes.c_int32),
        ("amgr_distance", ctypes.c_int32),
        ("amgr_interp_max", ctypes.c_int32),
        ("amgr_sym_ac", ctypes.c_int32),
        ("zmarch", ctypes.c_int32),
        ("sell", ctypes.c_int32),
        ("lambda_device", ctypes.c_int32),
    ]


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("use_x0", ctypes.c_int32),
        ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int32),
        ("finest_hat", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("preconditioner", ctypes.c_int32),
        ("tune", ctypes.c_int32),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("outer_iters", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("relres", ctypes.POINTER(ctypes.c_double)),
    ]


class ProfRecord(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_char * 80),
        ("role", ctypes.c_char * 64),
        ("level", ctypes.c_int32),
        ("phase", ctypes.c_int32),
        ("bytes", ctypes.c_int64),
        ("us", ctypes.c_double),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with paper_2407_05930_gb300.build.build() "
            "(there is no CPU fallback)"
        )
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pi64 = ctypes.POINTER(i64)
    pi32 = ctypes.POINTER(i32)
    pdbl = ctypes.POINTER(dbl)
    sig = {
        "amgsym_opts_default": (None, [ctypes.POINTER(Opts)]),
        "amgsym_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
        "amgsym_last_error": (ctypes.c_char_p, []),
        "amgsym_create_problem": (i32, [i64, pi64, pi32, pdbl, i32, pi32, ctypes.POINTER(P)]),
        "amgsym_update_values": (i32, [P, pdbl]),
        "amgsym_problem_sizes": (i32, [P, pi64, pi64, pi32, pi64, pi64, pi64]),
        "amgsym_get_inner_block": (i32, [P, pi64, pi32, pdbl]),
        "amgsym_get_interface": (i32, [P, pi32, pi32, pdbl]),
        "amgsym_setup": (i32, [P, ctypes.POINTER(Opts)]),
        "amgsym_num_levels": (i32, [P]),
        "amgsym_level_sizes": (i32, [P, i32, pi64, pi64, pi64, pi64, pi64, pdbl]),
        "amgsym_get_level_matrix": (i32, [P, i32, i32, pi64, pi32, pdbl]),
        "amgsym_level_dia": (i32, [P, i32, i32, pi32, pi32, pi32]),
        "amgsym_cycle_timeout_check": (i32, [P, i32, i32, P]),
        "amgsym_profile_step": (i32, [P, P, P, i32, i64, i32, i32, i32, P, ctypes.POINTER(ProfRecord), i32, pi32]),
        "amgsym_solve": (i32, [P, P, P, i32, i64, ctypes.POINTER(SolveOpts), P, ctypes.POINTER(SolveInfo)]),
        "amgsym_solve_adjoint": (i32, [P, P, P, i32, i64, ctypes.POINTER(SolveOpts), P, ctypes.POINTER(SolveInfo)]),
        "amgsym_transform_forward": (i32, [P, P, i32, i64, P, P]),
        "amgsym_transform_backward": (i32, [P, P, i32, P, i64, P]),
        "amgsym_apply_reduced": (i32, [P, P, P, i32, i32, P]),
        "amgsym_vcycle": (i32, [P, P, P, i32, i32, i32, P]),
        "amgsym_vcycle_noalloc": (i32, [P, P, P, i32, i32, i32, P]),
        "amgsym_grid_widths": (i32, [i64, dbl, pdbl]),
        "amgsym_fv_nnz": (i64, [i32, pi64]),
        "amgsym_fv_assemble": (i32, [i32, pi64, pdbl, pdbl, pi64, pi32, pdbl]),
        "amgsym_fv_assemble_bc": (i32, [i32, pi64, pdbl, pdbl, i32, pi64, pi32, pdbl]),
        "amgsym_is_singular": (i32, [P]),
        "amgsym_lrc_setup": (i32, [P, i32, i32, ctypes.c_double, ctypes.c_uint64, P]),
        "amgsym_amgr_apply": (i32, [P, P, P, i32, i32, P]),
        "amgsym_lrcfsai_setup": (i32, [P, i32, i32, ctypes.c_double, ctypes.c_uint64, P]),
        "amgsym_lrcfsai_values": (i32, [P, pdbl]),
        "amgsym_solve_fsai": (i32, [P, P, P, i32, i64, ctypes.POINTER(SolveOpts), i32, P, ctypes.POINTER(SolveInfo)]),
        "amgsym_amgr_info": (i32, [P, pi64, pi64, pi64, pi32, ctypes.POINTER(ctypes.c_int8)]),
        "amgsym_amgr_matrix": (i32, [P, i32, pi64, pi32, pdbl]),
        "amgsym_lrc_values": (i32, [P, pdbl]),
        "amgsym_solve_gmres": (i32, [P, P, P, i32, i64, ctypes.POINTER(SolveOpts), i32, i32, P,
                                     ctypes.POINTER(SolveInfo)]),
        "amgsym_mirror_perm": (i32, [i32, pi64, i32, pi32]),
        "amgsym_fv_grad_logk": (i32, [i32, pi64, P, P, P, P, i32, i64, P, i32, P]),
        "amgsym_kernel_launches": (i64, []),
        "amgsym_get_tiles": (i32, [P, i32, i32, pi32, i32]),
        "amgsym_batch_create": (i32, [ctypes.POINTER(P), i32, pi32, ctypes.POINTER(P)]),
        "amgsym_batch_solve": (i32, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(SolveOpts), P,
                                     ctypes.POINTER(SolveInfo)]),
        "amgsym_batch_destroy": (None, [P]),
        "amgsym_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

#: C-ABI entry points declared in include/amgsym.h
EXPORTED = [
    name
    for name in (
        "amgsym_opts_default amgsym_solve_opts_default amgsym_last_error amgsym_create_problem amgsym_update_values "
        "amgsym_problem_sizes amgsym_get_inner_block amgsym_get_interface amgsym_setup "
        "amgsym_num_levels amgsym_level_sizes amgsym_get_level_matrix amgsym_solve "
        "amgsym_solve_adjoint amgsym_transform_forward amgsym_transform_backward "
        "amgsym_apply_reduced amgsym_vcycle amgsym_vcycle_noalloc amgsym_grid_widths amgsym_fv_nnz "
        "amgsym_fv_assemble amgsym_mirror_perm amgsym_fv_grad_logk amgsym_kernel_launches amgsym_destroy "
        "amgsym_batch_create amgsym_batch_solve amgsym_batch_destroy amgsym_get_tiles amgsym_level_dia "
        "amgsym_cycle_timeout_check amgsym_profile_step amgsym_fv_assemble_bc amgsym_is_singular "
        "amgsym_lrc_setup amgsym_lrc_values amgsym_solve_gmres amgsym_amgr_apply amgsym_amgr_info "
        "amgsym_amgr_matrix amgsym_lrcfsai_setup amgsym_lrcfsai_values amgsym_solve_fsai"
    ).split()
]


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib.amgsym_kernel_launches())


def _check(code: int):
    if code < 0:
        raise AmgsymError(code, lib.amgsym_last_error().decode())
    return code


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_opts(**kw) -> Opts:
    o = Opts()
    lib.amgsym_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown setup option {k}")
        setattr(o, k, v)
    return o


def default_solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib.amgsym_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown solve option {k}")
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------------------
# structured-grid generator (host)

def grid_widths(N: int, gamma: float) -> np.ndarray:
    w = np.empty(int(N), dtype=np.float64)
    _check(lib.amgsym_grid_widths(int(N), float(gamma), _ptr(w, ctypes.c_double)))
    return w


def fv_assemble(N, widths, k, bc: str = "dirichlet"):
    """Full operator of the structured grid: (rowptr int64, colidx int32, vals f64);
    bc "dirichlet" or "neumann" on every wall."""
    N = np.ascontiguousarray(N, dtype=np.int64)
    d = N.size
    nnz = lib.amgsym_fv_nnz(d, _ptr(N, ctypes.c_int64))
    n = int(np.prod(N))
    W = np.ascontiguousarray(np.concatenate([np.asarray(w, dtype=np.float64) for w in widths]))
    k = np.ascontiguousarray(k, dtype=np.float64)
    if k.size != n:
        raise ValueError("k must have one value per cell")
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    _check(lib.amgsym_fv_assemble_bc(d, _ptr(N, ctypes.c_int64), _ptr(W, ctypes.c_double), _ptr(k, ctypes.c_double),
                                     BC[bc], _ptr(rowptr, ctypes.c_int64), _ptr(col, ctypes.c_int32),
                                     _ptr(val, ctypes.c_double)))
    return rowptr, col, val


def mirror_perm(N, s: int) -> np.ndarray:
    N = np.ascontiguousarray(N, dtype=np.int64)
    n = int(np.prod(N))
    perm = np.empty(n, dtype=np.int32)
    _check(lib.amgsym_mirror_perm(N.size, _ptr(N, ctypes.c_int64), int(s), _ptr(perm, ctypes.c_int32)))
    return perm.reshape(1 << s, n >> s)


@dataclass
class SolveResult:
    iters: int
    outer_iters: int
    converged: bool
    relres: np.ndarray
    status: str


class Problem:
    """A created problem (``amgsym_create_problem``) and, after ``setup``,
    its AMG hierarchy on the device."""

    def __init__(self, n, rowptr, colidx, vals, s, perm):
        self._h = ctypes.c_void_p()
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        _check(lib.amgsym_create_problem(int(n), _ptr(rowptr, ctypes.c_int64), _ptr(colidx, ctypes.c_int32),
                                         _ptr(vals, ctypes.c_double), int(s), _ptr(perm, ctypes.c_int32),
                                         ctypes.byref(self._h)))
        self.n = int(n)
        self.s = int(s)
        self.nb = 1 << self.s
        self.n_b = self.n >> self.s
        self.grid = None

    @classmethod
    def structured(cls, N, gamma: float = 0.0, logk: Optional[np.ndarray] = None, s: int = 0,
                   bc: str = "dirichlet"):
        """Unit-cube finite-volume problem with N cells per axis and s mirror
        symmetries; bc "dirichlet" or "neumann" (the paper's model problem)."""
        N = tuple(int(v) for v in N)
        widths = [grid_widths(n, gamma) for n in N]
        n = int(np.prod(N))
        k = np.ones(n) if logk is None else np.exp(np.asarray(logk, dtype=np.float64))
        rowptr, col, val = fv_assemble(N, widths, k, bc)
        perm = mirror_perm(N, s)
        p = cls(n, rowptr, col, val, s, perm)
        p.grid = dict(N=N, widths=widths, k=k, bc=bc)
        return p

    @property
    def singular(self) -> bool:
        """Every row sums to zero (pure Neumann): see amgsym_is_singular."""
        return lib.amgsym_is_singular(self._h) == 1

    def close(self):
        if self._h:
            lib.amgsym_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- host
    def sizes(self):
        n, n_b, nnz, nir, nie = (ctypes.c_int64() for _ in range(5))
        s = ctypes.c_int32()
        _check(lib.amgsym_problem_sizes(self._h, ctypes.byref(n), ctypes.byref(n_b), ctypes.byref(s),
                                        ctypes.byref(nnz), ctypes.byref(nir), ctypes.byref(nie)))
        return dict(n=n.value, n_b=n_b.value, s=s.value, nnz_inn=nnz.value, n_iface_rows=nir.value,
                    n_iface_entries=nie.value)

    def inner_block(self):
        sz = self.sizes()
        rp = np.empty(sz["n_b"] + 1, dtype=np.int64)
        ci = np.empty(sz["nnz_inn"], dtype=np.int32)
        v = np.empty(sz["nnz_inn"], dtype=np.float64)
        _check(lib.amgsym_get_inner_block(self._h, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32),
                                          _ptr(v, ctypes.c_double)))
        return rp, ci, v

    def interface(self):
        sz = self.sizes()
        ne = sz["n_iface_entries"]
        r = np.empty(max(ne, 1), dtype=np.int32)
        c = np.empty(max(ne, 1), dtype=np.int32)
        v = np.empty(max(ne, 1) * self.nb, dtype=np.float64)
        _check(lib.amgsym_get_interface(self._h, _ptr(r, ctypes.c_int32), _ptr(c, ctypes.c_int32),
                                        _ptr(v, ctypes.c_double)))
        return r[:ne], c[:ne], v[: ne * self.nb].reshape(ne, self.nb)

    def update_values(self, vals):
        """New FP64 values for the pattern given at creation (amgsym_update_values);
        the hierarchy is released: call setup() again before solving."""
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        _check(lib.amgsym_update_values(self._h, _ptr(vals, ctypes.c_double)))
        return self

    def setup(self, **kw):
        o = default_opts(**kw)
        _check(lib.amgsym_setup(self._h, ctypes.byref(o)))
        return self

    def num_levels(self) -> int:
        return int(lib.amgsym_num_levels(self._h))

    def level_info(self, level: int):
        rows, nA, nP, cP, nG = (ctypes.c_int64() for _ in range(5))
        om = ctypes.c_double()
        _check(lib.amgsym_level_sizes(self._h, level, ctypes.byref(rows), ctypes.byref(nA), ctypes.byref(nP),
                                      ctypes.byref(cP), ctypes.byref(nG), ctypes.byref(om)))
        return dict(rows=rows.value, nnz_A=nA.value, nnz_P=nP.value, cols_P=cP.value, nnz_G=nG.value,
                    omega=om.value)

    def level_matrix(self, level: int, which: str):
        """Host CSR (rowptr, colidx, vals, shape) of A, P or G on a level."""
        info = self.level_info(level)
        w = {"A": 0, "P": 1, "G": 2}[which]
        rows = info["rows"]
        nnz = {"A": info["nnz_A"], "P": info["nnz_P"], "G": info["nnz_G"]}[which]
        cols = info["cols_P"] if which == "P" else rows
        rp = np.empty(rows + 1, dtype=np.int64)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        v = np.empty(max(nnz, 1), dtype=np.float64)
        _check(lib.amgsym_get_level_matrix(self._h, level, w, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32),
                                           _ptr(v, ctypes.c_double)))
        return rp, ci[:nnz], v[:nnz], (rows, cols)

    def level_dia(self, level: int, which: str):
        """Diagonal-offset form of A, G or Gt on a level: {'ndiag', 'nstored', 'offsets'}
        (ndiag = 0: CSR only)."""
        w = {"A": 0, "G": 2, "Gt": 3}[which]
        nd, ns = ctypes.c_int32(), ctypes.c_int32()
        off = np.zeros(8, dtype=np.int32)
        _check(lib.amgsym_level_dia(self._h, level, w, ctypes.byref(nd), ctypes.byref(ns), _ptr(off, ctypes.c_int32)))
        return dict(ndiag=nd.value, nstored=ns.value, offsets=[int(v) for v in off[: nd.value]])

    # ---------------------------------------------------------------- device
    @staticmethod
    def _stream():
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def solve(self, b, x=None, adjoint: bool = False, **kw) -> SolveResult:
        """Solve A x = b.  b: CUDA float64 tensor [n] or [nrhs, n] (natural order).
        x: optional output tensor of the same shape (initial guess with use_x0=1)."""
        import torch

        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.float64):
            raise TypeError("b must be a CUDA float64 tensor")
        bb = b.reshape(-1, self.n)
        if not bb.is_contiguous():
            bb = bb.contiguous()
        nrhs = bb.shape[0]
        if x is None:
            x = torch.empty_like(bb)
        xx = x.reshape(-1, self.n)
        o = default_solve_opts(**kw)
        rel = np.zeros(nrhs, dtype=np.float64)
        info = SolveInfo()
        info.relres = _ptr(rel, ctypes.c_double)
        fn = lib.amgsym_solve_adjoint if adjoint else lib.amgsym_solve
        code = fn(self._h, ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(xx.data_ptr()), nrhs, self.n,
                  ctypes.byref(o), self._stream(), ctypes.byref(info))
        _check(code)
        res = SolveResult(info.iters, info.outer_iters, bool(info.converged), rel, STATUS[code])
        return x if x.shape == b.shape else xx.reshape(b.shape), res

    def amgr_info(self):
        """AMGR sizes and splitting (amgsym_amgr_info): dict n_cb, nnz_P, nnz_Ac, levels, cf."""
        ncb, nP, nA = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lev = ctypes.c_int32()
        cf = np.empty(self.n_b, dtype=np.int8)
        _check(lib.amgsym_amgr_info(self._h, ctypes.byref(ncb), ctypes.byref(nP), ctypes.byref(nA), ctypes.byref(lev),
                                    cf.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))))
        return dict(n_cb=ncb.value, nnz_P=nP.value, nnz_Ac=nA.value, levels=lev.value, cf=cf)

    def amgr_matrix(self, which: str):
        """Host CSR (rowptr, colidx, vals, shape) of P_b ("P") or A_c ("Ac")."""
        info = self.amgr_info()
        if which == "P":
            rows, cols, nnz, w = self.n_b, info["n_cb"], info["nnz_P"], 0
        else:
            rows = cols = info["n_cb"] * self.nb
            nnz, w = info["nnz_Ac"], 1
        rp = np.empty(rows + 1, dtype=np.int64)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        v = np.empty(max(nnz, 1), dtype=np.float64)
        _check(lib.amgsym_amgr_matrix(self._h, w, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32),
                                      _ptr(v, ctypes.c_double)))
        return rp, ci[:nnz], v[:nnz], (rows, cols)

    def amgr_apply(self, R, Z, nrhs: int, prec: int = PREC_FP64):
        _check(lib.amgsym_amgr_apply(self._h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr()), nrhs, prec,
                                     self._stream()))
        return Z

    @staticmethod
    def _ritz_steps(k: int, steps: Optional[int]) -> int:
        return int(steps) if steps is not None else max(40, 3 * int(k) + 8)

    def lrc_setup(self, k: int, steps: Optional[int] = None, tol: float = 0.1, seed: int = 7):
        """LRCAMG(k): the k smallest eigenpairs of M_inn^{-1} A^_i per block (amgsym_lrc_setup);
        steps = the restarted Lanczos basis size (default max(40, 3k + 8))."""
        _check(lib.amgsym_lrc_setup(self._h, int(k), self._ritz_steps(k, steps), float(tol), int(seed),
                                    self._stream()))
        return self

    def lrc_values(self) -> np.ndarray:
        """Ritz values [2^s, k] of the low-rank correction (empty without one)."""
        k = lib.amgsym_lrc_values(self._h, None)
        if k <= 0:
            return np.zeros((self.nb, 0))
        out = np.empty(self.nb * k, dtype=np.float64)
        lib.amgsym_lrc_values(self._h, _ptr(out, ctypes.c_double))
        return out.reshape(self.nb, k)

    def lrcfsai_setup(self, k: int, steps: Optional[int] = None, tol: float = 0.1, seed: int = 7):
        """LRCFSAI(k): the k smallest eigenpairs of G_inn A^_i G_inn^T per block (amgsym_lrcfsai_setup)."""
        _check(lib.amgsym_lrcfsai_setup(self._h, int(k), self._ritz_steps(k, steps), float(tol), int(seed),
                                        self._stream()))
        return self

    def lrcfsai_values(self) -> np.ndarray:
        k = lib.amgsym_lrcfsai_values(self._h, None)
        if k <= 0:
            return np.zeros((self.nb, 0))
        out = np.empty(self.nb * k, dtype=np.float64)
        lib.amgsym_lrcfsai_values(self._h, _ptr(out, ctypes.c_double))
        return out.reshape(self.nb, k)

    def solve_fsai(self, b, x=None, lrc: bool = False, **kw) -> SolveResult:
        """PCG with I (x) G_inn^T G_inn, optionally LRCFSAI-corrected (amgsym_solve_fsai); FP64."""
        import torch

        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.float64):
            raise TypeError("b must be a CUDA float64 tensor")
        bb = b.reshape(-1, self.n).contiguous()
        nrhs = bb.shape[0]
        if x is None:
            x = torch.empty_like(bb)
        xx = x.reshape(-1, self.n)
        o = default_solve_opts(**kw)
        rel = np.zeros(nrhs, dtype=np.float64)
        info = SolveInfo()
        info.relres = _ptr(rel, ctypes.c_double)
        code = lib.amgsym_solve_fsai(self._h, ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(xx.data_ptr()), nrhs,
                                     self.n, ctypes.byref(o), 1 if lrc else 0, self._stream(), ctypes.byref(info))
        _check(code)
        res = SolveResult(info.iters, info.outer_iters, bool(info.converged), rel, STATUS[code])
        return (x if x.shape == b.shape else xx.reshape(b.shape)), res

    def solve_gmres(self, b, x=None, restart: int = 30, lrc: bool = False, **kw) -> SolveResult:
        """Restarted GMRES with the LRCAMG preconditioner (amgsym_solve_gmres); FP64."""
        import torch

        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.float64):
            raise TypeError("b must be a CUDA float64 tensor")
        bb = b.reshape(-1, self.n).contiguous()
        nrhs = bb.shape[0]
        if x is None:
            x = torch.empty_like(bb)
        xx = x.reshape(-1, self.n)
        o = default_solve_opts(**kw)
        rel = np.zeros(nrhs, dtype=np.float64)
        info = SolveInfo()
        info.relres = _ptr(rel, ctypes.c_double)
        code = lib.amgsym_solve_gmres(self._h, ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(xx.data_ptr()), nrhs,
                                      self.n, ctypes.byref(o), int(restart), 1 if lrc else 0, self._stream(),
                                      ctypes.byref(info))
        _check(code)
        res = SolveResult(info.iters, info.outer_iters, bool(info.converged), rel, STATUS[code])
        return (x if x.shape == b.shape else xx.reshape(b.shape)), res

    def solve_async(self, b, x, nrhs: int, **kw) -> int:
        """Launch a solve without reading back its info (no host synchronisation
        beyond the convergence checks); returns the status code."""
        o = default_solve_opts(**kw)
        return _check(lib.amgsym_solve(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs,
                                       self.n, ctypes.byref(o), self._stream(), None))

    def transform_forward(self, b, nrhs: int, out):
        _check(lib.amgsym_transform_forward(self._h, ctypes.c_void_p(b.data_ptr()), nrhs, self.n,
                                            ctypes.c_void_p(out.data_ptr()), self._stream()))
        return out

    def transform_backward(self, xhat, nrhs: int, out):
        _check(lib.amgsym_transform_backward(self._h, ctypes.c_void_p(xhat.data_ptr()), nrhs,
                                             ctypes.c_void_p(out.data_ptr()), self.n, self._stream()))
        return out

    def apply_reduced(self, X, Y, nrhs: int, prec: int = PREC_FP64):
        _check(lib.amgsym_apply_reduced(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                        nrhs, prec, self._stream()))
        return Y

    def tiles(self, nrhs: int = 1, prec: int = PREC_MIXED_FP32, max_levels: int = 16):
        """SpMM tiles (columns per thread, entry lanes) in use: {'K3': (..), 'levels': [{A,G,Gt,R,P}]}."""
        out = np.zeros(2 + 10 * max_levels, dtype=np.int32)
        _check(lib.amgsym_get_tiles(self._h, nrhs, prec, _ptr(out, ctypes.c_int32), max_levels))
        levels = []
        for l in range(max_levels):
            v = out[2 + 10 * l: 12 + 10 * l].reshape(5, 2)
            if not v.any():
                break
            levels.append({k: tuple(int(t) for t in v[i]) for i, k in enumerate(["A", "G", "Gt", "R", "P"])})
        return {"K3": (int(out[0]), int(out[1])), "levels": levels}

    def vcycle_noalloc(self, R, Z, nrhs: int, prec: int = PREC_FP64, finest_hat: bool = False):
        """The V-cycle with its work vectors in the library's fixed device
        scratch (no allocation); see amgsym_vcycle_noalloc in include/amgsym.h."""
        _check(lib.amgsym_vcycle_noalloc(self._h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                                         nrhs, prec, 1 if finest_hat else 0, self._stream()))
        return Z

    def profile_step(self, b, x, nrhs: int, prec: int = PREC_MIXED_FP32, finest_hat: bool = False,
                     max_records: int = 512, preconditioner: int = PC_AMG):
        """Event-timed launches of one solve step (amgsym_profile_step): a list of
        dicts with kernel, role, level, phase (1 = every PCG iteration), bytes, us."""
        recs = (ProfRecord * max_records)()
        cnt = ctypes.c_int32()
        _check(lib.amgsym_profile_step(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs,
                                       self.n, prec, 1 if finest_hat else 0, int(preconditioner), self._stream(),
                                       recs, max_records,
                                       ctypes.byref(cnt)))
        return [dict(kernel=r.kernel.decode(), role=r.role.decode(), level=r.level, phase=r.phase, bytes=r.bytes,
                     us=r.us) for r in recs[: min(cnt.value, max_records)]]

    def cycle_timeout_check(self, nrhs: int = 1, prec: int = PREC_MIXED_FP32):
        """Run the persistent coarse-cycle kernel with a barrier nothing releases
        (see amgsym_cycle_timeout_check); raises unless the timeout was reported."""
        _check(lib.amgsym_cycle_timeout_check(self._h, nrhs, prec, self._stream()))

    def vcycle(self, R, Z, nrhs: int, prec: int = PREC_FP64, finest_hat: bool = False):
        _check(lib.amgsym_vcycle(self._h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr()), nrhs, prec,
                                 1 if finest_hat else 0, self._stream()))
        return Z


class Batch:
    """Many set-up problems solved together (``amgsym_batch_create`` /
    ``amgsym_batch_solve``): one persistent work-list launch per step of the
    inner PCG for all problems, one CUDA-graph replay per iteration."""

    def __init__(self, problems, nrhs):
        self.problems = list(problems)  # keep the problems alive
        self.nrhs = [int(v) for v in nrhs]
        if len(self.nrhs) != len(self.problems):
            raise ValueError("one nrhs per problem")
        arr = (ctypes.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        nr = np.ascontiguousarray(self.nrhs, dtype=np.int32)
        self._h = ctypes.c_void_p()
        _check(lib.amgsym_batch_create(arr, len(self.problems), _ptr(nr, ctypes.c_int32), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib.amgsym_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, xs=None, **kw):
        """bs: list of CUDA float64 tensors [nrhs_p, n_p]; returns (xs, results)."""
        import torch

        n = len(self.problems)
        bs = [b.reshape(self.nrhs[p], self.problems[p].n).contiguous() for p, b in enumerate(bs)]
        if xs is None:
            xs = [torch.empty_like(b) for b in bs]
        kw.setdefault("precision", PREC_MIXED_FP32)
        o = default_solve_opts(**kw)
        rel = [np.zeros(self.nrhs[p], dtype=np.float64) for p in range(n)]
        infos = (SolveInfo * n)()
        for p in range(n):
            infos[p].relres = _ptr(rel[p], ctypes.c_double)
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        code = lib.amgsym_batch_solve(self._h, bp, xp, ctypes.byref(o),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), infos)
        _check(code)
        res = [SolveResult(infos[p].iters, infos[p].outer_iters, bool(infos[p].converged), rel[p], STATUS[code])
               for p in range(n)]
        return xs, res


def fv_grad_logk(N, widths_dev, k_dev, u_dev, lam_dev, grad_dev, nrhs: int = 1, accumulate: bool = False):
    """Adjoint coefficient gradient on the device (see include/amgsym.h)."""
    import torch

    N = np.ascontiguousarray(N, dtype=np.int64)
    n = int(np.prod(N))
    _check(lib.amgsym_fv_grad_logk(N.size, _ptr(N, ctypes.c_int64), ctypes.c_void_p(widths_dev.data_ptr()),
                                   ctypes.c_void_p(k_dev.data_ptr()), ctypes.c_void_p(u_dev.data_ptr()),
                                   ctypes.c_void_p(lam_dev.data_ptr()), nrhs, n, ctypes.c_void_p(grad_dev.data_ptr()),
                                   1 if accumulate else 0,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return grad_dev
