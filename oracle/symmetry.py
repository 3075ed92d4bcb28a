"""Mirrored ordering of a structured grid and the block structure it induces.

ORACLE (test infrastructure only; see ``oracle/__init__.py``).

Sec. 2, eq. "fields_struct" and Fig. "1d_case": with one reflection
symmetry the unknowns of one half are numbered first, then those of the other
half with the *mirrored* local numbering, so mirror images share a local
index.  Applied recursively for ``s`` symmetries (eq. "struct_2sym") this
gives ``2^s`` copies of the base mesh.

Reading used throughout (the paper fixes no axis or copy order):

* symmetry ``b`` (0-based) reflects grid axis ``b`` (x, then y, then z) about
  the domain mid-plane;
* copy ``j`` (0-based) is the base octant reflected across every axis ``b``
  whose bit ``b`` is set in ``j``; copy 0 is the all-lower octant;
* the base octant is numbered lexicographically, x fastest; copy ``j``'s
  local index ``l`` is the cell whose coordinates along the reflected axes are
  ``i_b -> N_b - 1 - i_b``.

``perm[j, l]`` is the natural (x-fastest) index of local cell ``l`` of copy
``j``.  With this map the coupling of copy ``p`` to copy ``q`` is the block
``H_{p XOR q}`` (the dyadic pattern of eq. "struct_2sym").
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def base_shape(N, s: int):
    N = tuple(int(v) for v in N)
    if s > len(N):
        raise ValueError("more symmetries than axes")
    M = list(N)
    for b in range(s):
        if N[b] % 2:
            raise ValueError("a mirrored axis needs an even number of cells")
        M[b] = N[b] // 2
    return tuple(M)


def mirror_perm(N, s: int) -> np.ndarray:
    """``perm`` of shape ``(2^s, n/2^s)`` (int64), written cell by cell from
    the definition above with plain Python loops over the base cells' axes."""
    N = tuple(int(v) for v in N)
    d = len(N)
    M = base_shape(N, s)
    nb = 1 << s
    n_b = int(np.prod(M))
    perm = np.empty((nb, n_b), dtype=np.int64)
    # Base coordinates of every local index l (x fastest).
    coords = np.indices(M[::-1]).reshape(d, -1)[::-1]  # coords[a][l]
    for j in range(nb):
        c = coords.copy()
        for b in range(s):
            if (j >> b) & 1:
                c[b] = N[b] - 1 - c[b]
        nat = np.zeros(n_b, dtype=np.int64)
        stride = 1
        for a in range(d):
            nat += c[a] * stride
            stride *= N[a]
        perm[j] = nat
    return perm


def mirror_perm_bruteforce(N, s: int) -> np.ndarray:
    """The same map with explicit Python loops (for tiny grids only)."""
    N = tuple(int(v) for v in N)
    d = len(N)
    M = base_shape(N, s)
    nb = 1 << s
    out = []
    for j in range(nb):
        row = []
        for l in range(int(np.prod(M))):
            rem = l
            c = []
            for a in range(d):
                c.append(rem % M[a])
                rem //= M[a]
            for b in range(s):
                if (j >> b) & 1:
                    c[b] = N[b] - 1 - c[b]
            nat = 0
            stride = 1
            for a in range(d):
                nat += c[a] * stride
                stride *= N[a]
            row.append(nat)
        out.append(row)
    return np.array(out, dtype=np.int64)


def mirror_order(perm: np.ndarray) -> np.ndarray:
    """Flat gather index: ``x_mirror = x_natural[mirror_order(perm)]`` stacks
    the copies ``(x_1; ...; x_{2^s})`` as in eq. "fields_struct"."""
    return perm.reshape(-1)


def blocks(A: sp.spmatrix, perm: np.ndarray):
    """``H_m`` = coupling of copy 0 with copy ``m`` (eq. "struct_2sym"),
    ``m = 0 .. 2^s-1``; ``H_0`` is the inner block ``H_inn`` of eq. "split_s"."""
    A = sp.csr_matrix(A)
    r0 = perm[0]
    return [sp.csr_matrix(A[r0, :][:, perm[m]]) for m in range(perm.shape[0])]


def check_dyadic_structure(A: sp.spmatrix, perm: np.ndarray) -> float:
    """Largest ``|A[perm[p], perm[q]] - H_{p XOR q}|`` over all copy pairs
    (dense, tiny grids only)."""
    Ad = sp.csr_matrix(A).toarray()
    H = [Ad[np.ix_(perm[0], perm[m])] for m in range(perm.shape[0])]
    worst = 0.0
    nb = perm.shape[0]
    for p in range(nb):
        for q in range(nb):
            blk = Ad[np.ix_(perm[p], perm[q])]
            worst = max(worst, float(np.max(np.abs(blk - H[p ^ q]))) if blk.size else 0.0)
    return worst
