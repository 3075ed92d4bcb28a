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
"""

from __future__ import annotations

import numpy as np
import torch

from . import PREC_FP64, Problem, fv_grad_logk


class SymPoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, logk, N, gamma, s, solve_kw, setup_kw):
        N = tuple(int(v) for v in N)
        g_host = logk.detach().to("cpu", torch.float64).numpy()
        P = Problem.structured(N, gamma, g_host, s).setup(**(setup_kw or {}))
        u, info = P.solve(b.detach().contiguous(), **(solve_kw or {}))
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info}")
        ctx.P = P
        ctx.N = N
        ctx.solve_kw = solve_kw or {}
        widths = torch.from_numpy(np.concatenate(P.grid["widths"])).to(b.device)
        k = torch.from_numpy(P.grid["k"]).to(b.device)
        ctx.save_for_backward(u, widths, k)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, gu):
        u, widths, k = ctx.saved_tensors
        P = ctx.P
        lam, info = P.solve(gu.contiguous(), adjoint=True, **ctx.solve_kw)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge: {info}")
        nrhs = u.numel() // P.n
        grad_g = torch.empty(P.n, dtype=torch.float64, device=u.device)
        fv_grad_logk(ctx.N, widths, k, u.contiguous(), lam.contiguous(), grad_g, nrhs=nrhs)
        return lam, grad_g, None, None, None, None, None


def sym_poisson_solve(b, logk, N, gamma: float = 0.0, s: int = 0, solve_kw=None, setup_kw=None):
    """``u = A(exp(logk))^{-1} b``; differentiable in ``b`` and ``logk``.

    b: CUDA float64 ``[n]`` or ``[nrhs, n]`` (natural order, x fastest);
    logk: float64 ``[n]`` per-cell log-coefficient, mirror-symmetric under the
    ``s`` reflections (checked by ``amgsym_create_problem``).
    """
    kw = dict(tol=1e-10, precision=PREC_FP64)
    kw.update(solve_kw or {})
    return SymPoissonSolve.apply(b, logk, tuple(N), float(gamma), int(s), kw, setup_kw)
