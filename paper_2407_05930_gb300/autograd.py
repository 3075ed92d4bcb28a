"""Differentiable symmetry-reduced Poisson solve (``torch.autograd.Function``).

Forward: ``u = A(k)^{-1} b`` on a structured unit-cube grid with ``k =
exp(g)`` mirror-symmetric, solved by the reduced AMG-PCG of Alg. 1.
Backward (hand-written adjoint): ``A`` is symmetric, so the adjoint system
``A lambda = dL/du`` is the same reduced solve (``amgsym_solve_adjoint``);
then ``dL/db = lambda`` and ``dL/dg`` comes from the face-by-face formula of
the finite-volume transmissibilities (``amgsym_fv_grad_logk``, a CUDA kernel):

    dL/dg_c = sum_{faces f of c} -(lam_p - lam_q)(u_p - u_q) * t_f^2 h_c / (2 area_f k_c)

(a boundary face has ``-lam_p u_p``).  The gradient is with respect to the
full per-cell field; it is exact at the symmetric point even for directions
that break the symmetry (the operator is only evaluated there).

In an optimisation loop the grid stays and only ``g`` changes.  A
``SymPoisson`` keeps one library handle for its grid: a new ``g`` is
assembled on the host and passed to ``amgsym_update_values`` (same pattern,
validated again) followed by ``amgsym_setup``; the same ``g`` as the last
forward reuses the hierarchy as it is.
"""

from __future__ import annotations

import numpy as np
import torch

from . import PREC_FP64, Problem, fv_assemble, fv_grad_logk, grid_widths


class SymPoisson:
    """The differentiable solve on one grid (N cells per axis, stretching
    gamma, s mirror symmetries), holding one problem handle across calls."""

    def __init__(self, N, gamma: float = 0.0, s: int = 0, solve_kw=None, setup_kw=None):
        self.N = tuple(int(v) for v in N)
        self.gamma = float(gamma)
        self.s = int(s)
        self.solve_kw = dict(tol=1e-10, precision=PREC_FP64)
        self.solve_kw.update(solve_kw or {})
        self.setup_kw = dict(setup_kw or {})
        self.widths = [grid_widths(n, self.gamma) for n in self.N]
        self.n = int(np.prod(self.N))
        self.P = None
        self._logk = None  # host copy of the field the hierarchy was built for
        self.creates = 0   # problems created (1 for the handle's life)
        self.setups = 0    # hierarchy builds
        self._dev = None   # (device, widths tensor, k tensor) of the current field

    def _problem(self, g_host: np.ndarray, device) -> Problem:
        if self.P is not None and self._logk is not None and np.array_equal(g_host, self._logk):
            return self.P
        k = np.exp(g_host)
        if self.P is None:
            self.P = Problem.structured(self.N, self.gamma, g_host, self.s)
            self.creates += 1
        else:
            _, _, vals = fv_assemble(self.N, self.widths, k)
            self.P.update_values(vals)
            self.P.grid = dict(N=self.N, widths=self.widths, k=k)
        self.P.setup(**self.setup_kw)
        self.setups += 1
        self._logk = g_host.copy()
        self._dev = (device, torch.from_numpy(np.concatenate(self.widths)).to(device),
                     torch.from_numpy(k).to(device))
        return self.P

    def __call__(self, b, logk):
        return _SymPoissonSolve.apply(b, logk, self)


class _SymPoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, logk, op):
        g_host = np.ascontiguousarray(logk.detach().to("cpu", torch.float64).numpy())
        if g_host.size != op.n:
            raise ValueError("logk must have one value per cell")
        P = op._problem(g_host, b.device)
        u, info = P.solve(b.detach().contiguous(), **op.solve_kw)
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info}")
        ctx.op = op
        ctx.g_host = g_host
        _, widths, k = op._dev
        ctx.save_for_backward(u, widths, k)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, gu):
        u, widths, k = ctx.saved_tensors
        # the operator of this forward (another forward on the same handle
        # may have set up a different field since)
        P = ctx.op._problem(ctx.g_host, u.device)
        lam, info = P.solve(gu.contiguous(), adjoint=True, **ctx.op.solve_kw)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge: {info}")
        nrhs = u.numel() // P.n
        grad_g = torch.empty(P.n, dtype=torch.float64, device=u.device)
        fv_grad_logk(ctx.op.N, widths, k, u.contiguous(), lam.contiguous(), grad_g, nrhs=nrhs)
        return lam, grad_g, None


_CACHE: dict = {}
_CACHE_MAX = 4  # handles kept (each holds its hierarchy on the device)


def sym_poisson_solve(b, logk, N, gamma: float = 0.0, s: int = 0, solve_kw=None, setup_kw=None):
    """``u = A(exp(logk))^{-1} b``; differentiable in ``b`` and ``logk``.

    b: CUDA float64 ``[n]`` or ``[nrhs, n]`` (natural order, x fastest);
    logk: float64 ``[n]`` per-cell log-coefficient, mirror-symmetric under the
    ``s`` reflections (checked by ``amgsym_create_problem`` /
    ``amgsym_update_values``).  Calls with the same grid, options and device
    share one ``SymPoisson`` (one problem handle).
    """
    key = (tuple(int(v) for v in N), float(gamma), int(s), tuple(sorted((solve_kw or {}).items())),
           tuple(sorted((setup_kw or {}).items())), str(b.device))
    op = _CACHE.pop(key, None)
    if op is None:
        op = SymPoisson(N, gamma, s, solve_kw, setup_kw)
    _CACHE[key] = op  # most recently used last
    while len(_CACHE) > _CACHE_MAX:
        _CACHE.pop(next(iter(_CACHE)))
    return op(b, logk)
