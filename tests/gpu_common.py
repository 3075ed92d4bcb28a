"""Shared helpers of the GPU parity tests: oracle-side reference values in
the library's interleaved layout.  Everything here calls only ``oracle`` and
``synth``; the CUDA path is called by the tests themselves."""

from __future__ import annotations

import numpy as np

from oracle import fv, symmetry, transform
from synth import gaussian_logk


def oracle_problem(N, s, gamma=0.0, vark=False, seed=3, corr=2.0):
    g = gaussian_logk(N, s, seed=seed, corr=corr) if vark else None
    h, k, A = fv.grid_operator(N, gamma, g)
    return g, h, k, A


def oracle_hat_blocks(A, N, s):
    perm = symmetry.mirror_perm(N, s)
    H = symmetry.blocks(A, perm)
    return perm, transform.hat_blocks_sparse(H)


def oracle_forward(b, N, s):
    """2^{s/2} P_s (mirror-ordered b) in the interleaved layout [n_b][nrhs*2^s]."""
    perm = symmetry.mirror_perm(N, s)
    order = symmetry.mirror_order(perm)
    b = np.atleast_2d(b)
    nrhs = b.shape[0]
    nb = 1 << s
    n_b = b.shape[1] // nb
    out = np.empty((n_b, nrhs * nb))
    for r in range(nrhs):
        y = transform.P_s_apply(s, b[r][order]) * 2.0 ** (s / 2.0)
        out[:, r * nb:(r + 1) * nb] = y.reshape(nb, n_b).T
    return out


def oracle_apply_hat(hat, X, nb):
    """Y[:, c] = A^_{c mod nb} X[:, c]."""
    Y = np.empty_like(X)
    for c in range(X.shape[1]):
        Y[:, c] = hat[c % nb] @ X[:, c]
    return Y
