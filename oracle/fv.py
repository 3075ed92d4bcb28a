"""Cell-centred finite-volume assembly of ``-div(k grad u) = f`` (ORACLE).

Test infrastructure only (see ``oracle/__init__.py``).

The paper discretises its model problem (Sec. 2.2, eq. "modelproblem") with
a standard 7-point stencil on the tanh-stretched unit cube.  The operator
here is the two-point-flux finite-volume Laplacian with homogeneous
Dirichlet conditions, written without division by the cell volume so that
it stays symmetric on stretched grids:

* interior face ``f`` between cells ``p`` and ``q`` along axis ``a``:
  ``t_f = area_f / (h_p/(2 k_p) + h_q/(2 k_q))``, the series conductance of
  the two half cells (distance-weighted harmonic mean of ``k``);
* boundary face of cell ``p``: ``t_f = area_f / (h_p/(2 k_p))`` (the
  Dirichlet value sits on the face);
* ``A_pq = -t_f`` and ``A_pp = sum of t_f over the faces of p``, the faces of
  each axis summed as one (low + high) pair before the axes are added.

Unknowns are in natural lexicographic order with x fastest.  The right-hand
side of a source density ``f`` is ``f`` times the cell volume.

``bc="neumann"`` gives the paper's model problem (Sec. 2.2, eq.
"modelproblem": homogeneous Neumann on every wall): the boundary faces carry
no flux, so their transmissibility drops out of the diagonal, every row sums
to zero and the constant vector spans the null space.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _broadcast_axis(v: np.ndarray, a: int, d: int) -> np.ndarray:
    """Reshape a per-axis vector so it broadcasts along grid axis ``a`` of a
    C-ordered array with axes reversed (numpy axis ``d-1-a``)."""
    shape = [1] * d
    shape[d - 1 - a] = v.size
    return v.reshape(shape)


def cell_volumes(h) -> np.ndarray:
    d = len(h)
    vol = np.ones([1] * d)
    for a in range(d):
        vol = vol * _broadcast_axis(h[a], a, d)
    return vol.reshape(-1)


def face_areas(h, a: int) -> np.ndarray:
    """Area of the faces normal to axis ``a`` for every cell (product of the
    widths of the other axes), as a full C-ordered array."""
    d = len(h)
    N = [x.size for x in h]
    area = np.ones(N[::-1])
    for b in range(d):
        if b != a:
            area = area * _broadcast_axis(h[b], b, d)
    return area


def transmissibilities(h, k: np.ndarray):
    """Per-axis face transmissibilities.

    Returns a list over axes ``a`` of ``(t_interior, t_low, t_high)``:
    ``t_interior`` has the grid shape shortened by one along axis ``a`` (face
    between cell ``i`` and ``i+1``); ``t_low``/``t_high`` are the boundary
    faces at ``i = 0`` and ``i = N_a - 1`` (grid shape with that axis of
    length 1).
    """
    d = len(h)
    N = [x.size for x in h]
    kk = np.asarray(k, dtype=np.float64).reshape(N[::-1])
    out = []
    for a in range(d):
        ax = d - 1 - a
        half_res = _broadcast_axis(h[a], a, d) / (2.0 * kk)  # h_p / (2 k_p)
        area = face_areas(h, a)
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, N[a] - 1)
        hi[ax] = slice(1, N[a])
        t_int = area[tuple(lo)] / (half_res[tuple(lo)] + half_res[tuple(hi)])
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = slice(0, 1)
        last[ax] = slice(N[a] - 1, N[a])
        t_low = area[tuple(first)] / half_res[tuple(first)]
        t_high = area[tuple(last)] / half_res[tuple(last)]
        out.append((t_int, t_low, t_high))
    return out


def _boundary_weight(bc: str) -> float:
    if bc == "dirichlet":
        return 1.0
    if bc == "neumann":
        return 0.0
    raise ValueError(f"unknown boundary condition {bc!r}")


def assemble(h, k: np.ndarray, bc: str = "dirichlet") -> sp.csr_matrix:
    """Full unreduced operator ``A`` (CSR, FP64, natural order, x fastest)."""
    wb = _boundary_weight(bc)
    d = len(h)
    N = [x.size for x in h]
    n = int(np.prod(N))
    idx = np.arange(n).reshape(N[::-1])
    T = transmissibilities(h, k)
    rows, cols, vals = [], [], []
    diag = np.zeros(N[::-1])
    for a in range(d):
        ax = d - 1 - a
        t_int, t_low, t_high = T[a]
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, N[a] - 1)
        hi[ax] = slice(1, N[a])
        p = idx[tuple(lo)].reshape(-1)
        q = idx[tuple(hi)].reshape(-1)
        t = t_int.reshape(-1)
        rows += [p, q]
        cols += [q, p]
        vals += [-t, -t]
        # Per-axis pair sum (low face + high face) of every cell.
        s_low = np.zeros(N[::-1])
        s_high = np.zeros(N[::-1])
        s_low[tuple(hi)] = t_int          # cell i+1 sees face (i, i+1) as its low face
        s_high[tuple(lo)] = t_int         # cell i sees it as its high face
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = slice(0, 1)
        last[ax] = slice(N[a] - 1, N[a])
        s_low[tuple(first)] = wb * t_low
        s_high[tuple(last)] = wb * t_high
        diag = diag + (s_low + s_high)
    allr = np.arange(n)
    rows.append(allr)
    cols.append(allr)
    vals.append(diag.reshape(-1))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A = A.tocsr()
    A.sort_indices()
    return A


def apply(h, k: np.ndarray, u: np.ndarray, bc: str = "dirichlet") -> np.ndarray:
    """Matrix-free ``A u`` from the face fluxes ``t_f (u_p - u_q)``; used for
    residual checks at sizes where assembling ``A`` is wasteful."""
    wb = _boundary_weight(bc)
    d = len(h)
    N = [x.size for x in h]
    U = np.asarray(u, dtype=np.float64).reshape(N[::-1])
    T = transmissibilities(h, k)
    out = np.zeros(N[::-1])
    for a in range(d):
        ax = d - 1 - a
        t_int, t_low, t_high = T[a]
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, N[a] - 1)
        hi[ax] = slice(1, N[a])
        flux = t_int * (U[tuple(lo)] - U[tuple(hi)])
        out[tuple(lo)] += flux
        out[tuple(hi)] -= flux
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = slice(0, 1)
        last[ax] = slice(N[a] - 1, N[a])
        out[tuple(first)] += wb * t_low * U[tuple(first)]
        out[tuple(last)] += wb * t_high * U[tuple(last)]
    return out.reshape(-1)


def grid_operator(N, gamma: float, logk: np.ndarray | None = None, bc: str = "dirichlet"):
    """Convenience: widths, k and assembled ``A`` for a unit-cube grid."""
    from .grid import widths

    h = widths(N, gamma)
    n = int(np.prod(N))
    k = np.ones(n) if logk is None else np.exp(logk)
    return h, k, assemble(h, k, bc)
