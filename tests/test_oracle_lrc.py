"""Pins of the oracle's low-rank correction (Sec. 2.2, Thm.
"correction_nonfact", eq. "LRC_AMG") on small split operators
A^_i = A_inn + A_out,i of the symmetry-reduced Poisson problem:

* the full-rank correction of a preconditioner reproduces A^_i^{-1};
* with the exact inverse of A_inn as the preconditioner, Y = -A_inn^{-1} A_out,i
  has the rank of A_out,i (the plane rows; eq. "rank"), so the correction
  of that rank is exact;
* the rank-k correction maps the k smallest eigenvalues of the
  preconditioned operator to 1 and leaves the others where they were.
"""

import numpy as np
import pytest

from oracle import fv, grid, lrc, symmetry, transform
from synth import gaussian_logk


def _blocks(N, s, seed=5):
    g = gaussian_logk(N, s, seed=seed, corr=2.0)
    A = fv.assemble(grid.widths(N, 1.5), np.exp(g))
    H = symmetry.blocks(A, symmetry.mirror_perm(N, s))
    hat = transform.hat_blocks_sparse(H)
    return H[0].toarray(), [h.toarray() for h in hat]


def _jacobi_like(Ainn):
    """A cheap SPD approximate inverse (two damped Jacobi sweeps as a
    polynomial): the preconditioner need not be exact for the theorem."""
    D = np.diag(1.0 / np.diag(Ainn))
    return 0.6 * D + 0.6 * D - 0.36 * D @ Ainn @ D


@pytest.mark.parametrize("N,s", [((8, 6, 4), 1), ((6, 6, 4), 2)])
def test_full_rank_correction_is_the_inverse(N, s):
    Ainn, hat = _blocks(N, s)
    B = _jacobi_like(Ainn)
    for Ai in hat:
        Ainv = lrc.exact_inverse_by_correction(Ai, B)
        assert np.linalg.norm(Ainv @ Ai - np.eye(Ai.shape[0])) <= 1e-8


@pytest.mark.parametrize("N,s", [((8, 6, 4), 1), ((6, 8, 4), 3)])
def test_correction_of_the_interface_rank_is_exact_with_an_exact_inner_solve(N, s):
    Ainn, hat = _blocks(N, s)
    Binv = np.linalg.inv(Ainn)
    for i, Ai in enumerate(hat):
        r = np.linalg.matrix_rank(Ai - Ainn)  # rank of A_out,i: its plane rows
        lam = np.sort(np.linalg.eigvals(Binv @ Ai).real)
        assert np.sum(np.abs(lam - 1.0) > 1e-10) <= r  # all other eigenvalues are 1
        # the nonzero part of Y's spectrum alone already gives the inverse
        Ainv = lrc.exact_inverse_by_correction(Ai, Binv)
        assert np.linalg.norm(Ainv @ Ai - np.eye(Ai.shape[0])) <= 1e-8
    # block 0 (every mirror plane Neumann-like: A_out,0 is negative
    # semidefinite) has its r non-unit eigenvalues below 1, so the rank-r
    # correction of the r smallest (eq. "LRC_AMG") is exact; the last block
    # (every plane with the doubled coupling) has them above 1
    r = np.linalg.matrix_rank(hat[0] - Ainn)
    P, lam_r = lrc.low_rank_corrected(hat[0], Binv, r)
    assert np.all(lam_r < 1.0)
    assert np.linalg.norm(P @ hat[0] - np.eye(Ainn.shape[0])) <= 1e-8
    assert np.sort(np.linalg.eigvals(Binv @ hat[-1]).real)[0] >= 1.0 - 1e-10


def test_rank_k_correction_moves_the_smallest_eigenvalues_to_one():
    Ainn, hat = _blocks((8, 6, 6), 1)
    B = _jacobi_like(Ainn)
    Ai = hat[0]
    lam = np.sort(np.linalg.eigvals(B @ Ai).real)
    k = 5
    P, lam_k = lrc.low_rank_corrected(Ai, B, k)
    assert np.allclose(lam_k, lam[:k], rtol=1e-10)
    mu = np.sort(np.linalg.eigvals(P @ Ai).real)
    assert np.sum(np.abs(mu - 1.0) <= 1e-8) >= k  # the k smallest moved to 1
    assert np.allclose(mu[:-k] if k else mu, np.sort(np.concatenate([lam[k:], np.ones(k)]))[:-k], rtol=1e-8)


def test_factored_correction_theorem():
    """Thm. "correction" with a factored approximate inverse: all pairs give
    A^{-1}; the rank-k correction moves the k smallest eigenvalues of the
    preconditioned operator to 1 (eq. "LRC")."""
    Ainn, hat = _blocks((8, 6, 4), 2)
    L = np.linalg.cholesky(Ainn)
    G = np.tril(np.linalg.inv(L))
    G = np.where(np.abs(G) >= 0.05 * np.abs(G).max(axis=1, keepdims=True), G, 0.0)  # a sparse approximation
    for Ai in hat:
        M, _ = lrc.factored_corrected(Ai, G)
        assert np.linalg.norm(M @ Ai - np.eye(Ai.shape[0])) <= 1e-8
        k = 6
        Mk, lam_k = lrc.factored_corrected(Ai, G, k)
        mu = np.sort(np.linalg.eigvals(Mk @ Ai).real)
        lam = np.sort(np.linalg.eigvalsh(G @ Ai @ G.T))
        assert np.allclose(lam_k, lam[:k], rtol=1e-10)
        assert np.sum(np.abs(mu - 1.0) <= 1e-8) >= k
        assert np.allclose(np.sort(np.concatenate([lam[k:], np.ones(k)])), mu, rtol=1e-8, atol=1e-12)
