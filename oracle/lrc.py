"""Low-rank corrections of a preconditioner (ORACLE; test infrastructure
only, see ``oracle/__init__.py``): Sec. 2.2, Thm. "correction_nonfact" and
eqs. "Ydef_AMG", "FRC_AMG", "LRC_AMG".

Dense linear algebra on small matrices, written from the statements:

* ``exact_inverse_by_correction(A, Binv)``: with ``Y = I - Binv A`` and its
  eigendecomposition ``Y = U Sigma V^T`` (right eigenvectors ``U``, left
  eigenvectors ``V``, biorthonormal ``V^T U = I``), the theorem gives
  ``A^{-1} = (I + U (Sigma^{-1} - V^T U)^{-1} V^T) Binv``; only the
  eigenpairs with ``sigma != 0`` contribute (the others add nothing), so the
  sum runs over the nonzero part of the spectrum of ``Y``;
* ``low_rank_corrected(A, Binv, k)``: the rank-k truncation of eq.
  "LRC_AMG", keeping the k smallest eigenvalues ``lambda`` of
  ``X = Binv A`` (``Sigma = I - Lambda``, ``Theta = (Sigma^{-1} - I)^{-1}``);
* ``factored_corrected(A, G, k)``: Thm. "correction" and eq. "LRC" for a
  factored approximate inverse ``G^T G``: with ``Y = I - G A G^T = V Sigma
  V^T``, ``A^{-1} = G^T G + G^T V Sigma (I - Sigma)^{-1} V^T G``; ``k = None``
  keeps every eigenpair (the exact inverse), else the k of the smallest
  eigenvalues of ``G A G^T``.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _eig_biorthonormal(X: np.ndarray):
    """Eigenvalues (ascending, real), right eigenvectors U and left
    eigenvectors V of X with V^T U = I.  X = Binv A with Binv and A SPD has
    a real positive spectrum (it is similar to Binv^{1/2} A Binv^{1/2})."""
    w, vl, vr = sla.eig(X, left=True, right=True)
    order = np.argsort(w.real)
    w, vl, vr = w.real[order], vl.real[:, order], vr.real[:, order]
    # scale the left vectors so that v_t^T u_t = 1 (distinct eigenvalues are
    # biorthogonal already; equal ones are orthogonalised by the eigensolver)
    G = vl.T @ vr
    vl = vl @ np.linalg.inv(G).T
    return w, vr, vl


def exact_inverse_by_correction(A: np.ndarray, Binv: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """A^{-1} through the full-rank correction of Thm. "correction_nonfact"."""
    n = A.shape[0]
    X = Binv @ A
    lam, U, V = _eig_biorthonormal(X)
    sigma = 1.0 - lam
    keep = np.abs(sigma) > tol * np.max(np.abs(sigma))
    U, V, sigma = U[:, keep], V[:, keep], sigma[keep]
    core = np.linalg.inv(np.diag(1.0 / sigma) - V.T @ U)
    return (np.eye(n) + U @ core @ V.T) @ Binv


def low_rank_corrected(A: np.ndarray, Binv: np.ndarray, k: int):
    """(P, lam): the preconditioner (I + U_k Theta_k V_k^T) Binv of eq.
    "LRC_AMG" with the k smallest eigenvalues lam of Binv A."""
    n = A.shape[0]
    lam, U, V = _eig_biorthonormal(Binv @ A)
    lam_k, U_k, V_k = lam[:k], U[:, :k], V[:, :k]
    theta = (1.0 - lam_k) / lam_k  # (Sigma^{-1} - I)^{-1} with Sigma = I - Lambda
    return (np.eye(n) + U_k @ np.diag(theta) @ V_k.T) @ Binv, lam_k


def factored_corrected(A: np.ndarray, G: np.ndarray, k=None):
    """(M, lam): G^T G + Z Theta Z^T with Z = G^T V (eqs. "LRC", "LRCFSAI") and
    the eigenvalues lam of G A G^T it corrects (all of them for k = None)."""
    X = G @ A @ G.T
    X = 0.5 * (X + X.T)
    lam, V = np.linalg.eigh(X)
    if k is not None:
        lam, V = lam[:k], V[:, :k]
    sigma = 1.0 - lam
    keep = np.abs(1.0 - sigma) > 0.0  # lambda != 0
    theta = np.zeros_like(sigma)
    theta[keep] = sigma[keep] / (1.0 - sigma[keep])
    Z = G.T @ V
    return G.T @ G + Z @ np.diag(theta) @ Z.T, lam
