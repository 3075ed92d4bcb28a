"""The change of basis ``P_s`` and the decoupled blocks (Sec. 2).

ORACLE (test infrastructure only; see ``oracle/__init__.py``).

Eq. "P_s": ``P_s = prod_{i=1..s} (I_{2^{i-1}} (x) (1/sqrt2)[[1, 1], [1, -1]] (x) I_{n/2^i})``
acting on the mirror-stacked vector ``(x_1; ...; x_{2^s})`` of
eq. "fields_struct".  It is orthonormal and an involution (``P_s^{-1} = P_s``)
and eq. "hL_s" states ``P_s A P_s^{-1} = blockdiag(A^_1, ..., A^_{2^s})``;
eq. "hL_splitting" splits each block as ``A^_i = A_inn + A_out,i``.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_H2 = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)


def P_s_dense(s: int, n: int) -> np.ndarray:
    """Dense ``P_s`` as the product of its ``s`` Kronecker factors (small ``n``)."""
    if n % (1 << s):
        raise ValueError("n must be divisible by 2^s")
    P = np.eye(n)
    for i in range(1, s + 1):
        F = np.kron(np.kron(np.eye(1 << (i - 1)), _H2), np.eye(n >> i))
        P = P @ F
    return P


def P_s_apply(s: int, x: np.ndarray) -> np.ndarray:
    """``P_s x`` for a mirror-stacked vector (or a stack of them along the last
    axis), applying the Kronecker factors one at a time: factor ``i`` mixes
    the two halves of every block of length ``n/2^{i-1}``."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[-1]
    if n % (1 << s):
        raise ValueError("n must be divisible by 2^s")
    lead = x.shape[:-1]
    y = x.reshape(-1, n).copy()
    for i in range(1, s + 1):
        m = n >> i
        z = y.reshape(y.shape[0], 1 << (i - 1), 2, m)
        a = z[:, :, 0, :].copy()
        b = z[:, :, 1, :].copy()
        z[:, :, 0, :] = (a + b) / np.sqrt(2.0)
        z[:, :, 1, :] = (a - b) / np.sqrt(2.0)
        y = z.reshape(y.shape[0], n)
    return y.reshape(*lead, n)


def decoupled_blocks_dense(A_mirror: np.ndarray, s: int):
    """Diagonal blocks of ``P_s A P_s`` (eq. "hL_s") and the largest
    off-diagonal-block entry (zero up to rounding when the symmetry holds)."""
    n = A_mirror.shape[0]
    nb = 1 << s
    m = n // nb
    P = P_s_dense(s, n)
    Ah = P @ A_mirror @ P
    blocks = [Ah[i * m:(i + 1) * m, i * m:(i + 1) * m].copy() for i in range(nb)]
    off = Ah.copy()
    for i in range(nb):
        off[i * m:(i + 1) * m, i * m:(i + 1) * m] = 0.0
    return blocks, float(np.max(np.abs(off))) if off.size else 0.0


def hadamard_sign(i: int, j: int) -> float:
    """Entry ``(i, j)`` of the Sylvester-Hadamard matrix ``2^{s/2} P_s`` on
    block indices: the product of the 2x2 factors' entries over the bits."""
    sgn = 1.0
    t = i & j
    while t:
        if t & 1:
            sgn = -sgn
        t >>= 1
    return sgn


def hat_blocks_sparse(H):
    """``A^_i = sum_j sign(i, j) H_j`` for the ``2^s`` blocks of the dyadic
    structure (the diagonal blocks of ``P_s A P_s``, derived from
    eqs. "struct_2sym" and "P_s"); pinned against ``decoupled_blocks_dense``."""
    nb = len(H)
    out = []
    for i in range(nb):
        acc = sp.csr_matrix(H[0].shape)
        for j in range(nb):
            acc = acc + hadamard_sign(i, j) * H[j]
        out.append(sp.csr_matrix(acc))
    return out


def interface_blocks(H):
    """``A_out,i = A^_i - A_inn`` (eq. "hL_splitting"), ``A_inn = H_0``."""
    Ah = hat_blocks_sparse(H)
    return [sp.csr_matrix(Ah[i] - H[0]) for i in range(len(H))]
