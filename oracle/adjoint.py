"""Loss and gradients of the differentiable Poisson solve (ORACLE).

Test infrastructure only (see ``oracle/__init__.py``).  The paper has no
adjoint; these are the plain definitions the GPU adjoint is checked against.

Forward map: ``u = A(k)^{-1} b`` with ``k = exp(g)`` per cell and ``A(k)``
the finite-volume operator of ``oracle.fv``.  Loss ``L = ||u - u_t||^2``.

* ``lambda = A^{-1} (2 (u - u_t))`` (``A`` is symmetric, so the adjoint
  system is the forward one);
* ``dL/db = lambda``;
* ``A = sum_f t_f e_f e_f^T`` with ``e_f = e_p - e_q`` for an interior face and
  ``e_f = e_p`` for a boundary face, so ``dL/dt_f = -(lambda^T e_f)(e_f^T u)``;
* ``t_f = area_f / sum_{c in f} h_c / (2 k_c)`` gives
  ``dt_f/dg_c = t_f^2 h_c / (2 area_f k_c)``, and
  ``dL/dg_c = sum_{f containing c} dL/dt_f * dt_f/dg_c``.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fv


def solve_full(h, k, b):
    """Direct sparse solve of the full system (sizes up to ~10^5 unknowns)."""
    A = fv.assemble(h, k).tocsc()
    return spla.spsolve(A, b)


def loss(h, logk, b, u_t) -> float:
    u = solve_full(h, np.exp(logk), b)
    return float(np.sum((u - u_t) ** 2))


def gradients(h, logk, b, u_t):
    """``(L, dL/db, dL/dg)`` by the adjoint formulas above."""
    d = len(h)
    N = [x.size for x in h]
    k = np.exp(logk)
    A = fv.assemble(h, k).tocsc()
    u = spla.spsolve(A, b)
    lam = spla.spsolve(A, 2.0 * (u - u_t))
    L = float(np.sum((u - u_t) ** 2))
    gg = grad_logk(h, k, u, lam)
    return L, lam, gg


def grad_logk(h, k, u, lam):
    """``dL/dg`` given forward solution ``u`` and adjoint ``lam``."""
    d = len(h)
    N = [x.size for x in h]
    K = np.asarray(k).reshape(N[::-1])
    U = np.asarray(u).reshape(N[::-1])
    Lm = np.asarray(lam).reshape(N[::-1])
    T = fv.transmissibilities(h, k)
    g = np.zeros(N[::-1])
    for a in range(d):
        ax = d - 1 - a
        t_int, t_low, t_high = T[a]
        area = fv.face_areas(h, a)
        hb = fv._broadcast_axis(h[a], a, d) * np.ones(N[::-1])
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, N[a] - 1)
        hi[ax] = slice(1, N[a])
        lo, hi = tuple(lo), tuple(hi)
        dL_dt = -(Lm[lo] - Lm[hi]) * (U[lo] - U[hi])
        g[lo] += dL_dt * t_int ** 2 * hb[lo] / (2.0 * area[lo] * K[lo])
        g[hi] += dL_dt * t_int ** 2 * hb[hi] / (2.0 * area[hi] * K[hi])
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = slice(0, 1)
        last[ax] = slice(N[a] - 1, N[a])
        first, last = tuple(first), tuple(last)
        g[first] += -Lm[first] * U[first] * t_low ** 2 * hb[first] / (2.0 * area[first] * K[first])
        g[last] += -Lm[last] * U[last] * t_high ** 2 * hb[last] / (2.0 * area[last] * K[last])
    return g.reshape(-1)
