"""Pins of the oracle's solvers and adjoint (CPU only).

Two independent exact routes (dense Cholesky and the DST-II closed form) pin
each other and the CG; finite differences pin the adjoint gradients.
"""

import numpy as np
import pytest

from oracle import adjoint, fv, solvers
from synth import gaussian_logk, rhs_uniform, u_target


@pytest.mark.parametrize("N", [(6, 4), (5, 3, 4), (8, 8, 2)])
def test_dst_equals_dense(N):
    h, k, A = fv.grid_operator(N, 0.0)
    b = rhs_uniform(A.shape[0], 2, config=99)
    x_dense = np.stack([solvers.dense_solve(A, bi) for bi in b])
    x_dst = solvers.dst_solve(N, b)
    assert np.max(np.abs(x_dst - x_dense)) <= 1e-12 * np.max(np.abs(x_dense))


def test_cg_equals_dense_variable_k_stretched():
    N = (10, 8, 6)
    g = gaussian_logk(N, 1, seed=3, corr=2.0)
    h, k, A = fv.grid_operator(N, 1.5, g)
    b = rhs_uniform(A.shape[0], 1, config=98)[0]
    x_dense = solvers.dense_solve(A, b)
    x_cg, info = solvers.cg(A, b, tol=1e-13, return_info=True)
    assert info["relres"] <= 1e-13
    assert np.linalg.norm(x_cg - x_dense) <= 1e-10 * np.linalg.norm(x_dense)


def test_cg_equals_dst_64x64():
    N = (64, 64)
    h, k, A = fv.grid_operator(N, 0.0)
    b = rhs_uniform(A.shape[0], 1, config=1)[0]
    x_cg, info = solvers.cg(A, b, tol=1e-13, return_info=True)
    x_dst = solvers.dst_solve(N, b)
    assert np.linalg.norm(x_cg - x_dst) <= 1e-10 * np.linalg.norm(x_dst)


def test_cg_zero_rhs():
    h, k, A = fv.grid_operator((4, 4), 0.0)
    x = solvers.cg(A, np.zeros(16))
    assert np.all(x == 0)


def _small_adjoint_case(N=(6, 4, 4), s=2, gamma=1.5):
    g = gaussian_logk(N, s, seed=21, corr=1.5)
    from oracle import grid

    h = grid.widths(N, gamma)
    n = int(np.prod(N))
    b = rhs_uniform(n, 1, config=5)[0]
    ut = u_target(n)
    return h, g, b, ut


def test_self_adjoint():
    h, g, b, ut = _small_adjoint_case()
    k = np.exp(g)
    c = np.random.default_rng(1).standard_normal(b.size)
    x1 = adjoint.solve_full(h, k, b)
    x2 = adjoint.solve_full(h, k, c)
    assert abs(x1 @ c - b @ x2) <= 1e-12 * abs(x1 @ c)


def test_adjoint_gradients_vs_central_differences():
    h, g, b, ut = _small_adjoint_case()
    L, dLdb, dLdg = adjoint.gradients(h, g, b, ut)
    rng = np.random.default_rng(8)
    eps = 1e-6
    for _ in range(2):
        v = rng.standard_normal(g.size)
        fd = (adjoint.loss(h, g + eps * v, b, ut) - adjoint.loss(h, g - eps * v, b, ut)) / (2 * eps)
        assert abs(fd - dLdg @ v) <= 1e-6 * max(abs(fd), 1e-300) + 1e-10
        w = rng.standard_normal(b.size)
        fd = (adjoint.loss(h, g, b + eps * w, ut) - adjoint.loss(h, g, b - eps * w, ut)) / (2 * eps)
        assert abs(fd - dLdb @ w) <= 1e-6 * abs(fd) + 1e-10
    # a single-cell perturbation of a boundary cell exercises the boundary faces
    e = np.zeros(g.size)
    e[0] = 1.0
    fd = (adjoint.loss(h, g + eps * e, b, ut) - adjoint.loss(h, g - eps * e, b, ut)) / (2 * eps)
    assert abs(fd - dLdg[0]) <= 1e-5 * abs(fd) + 1e-10


@pytest.mark.slow
def test_adjoint_fd_32cube():
    h, g, b, ut = _small_adjoint_case(N=(32, 32, 32), s=3)
    L, dLdb, dLdg = adjoint.gradients(h, g, b, ut)
    v = np.random.default_rng(12).standard_normal(g.size)
    eps = 1e-6
    fd = (adjoint.loss(h, g + eps * v, b, ut) - adjoint.loss(h, g - eps * v, b, ut)) / (2 * eps)
    assert abs(fd - dLdg @ v) <= 1e-6 * abs(fd)


def test_lanczos_condition_estimate_bounds_true_condition():
    # the CG-Lanczos Ritz values lie inside the spectrum; for a small matrix
    # and enough iterations they converge to the extremes
    h, k, A = fv.grid_operator((12, 10), 0.0)
    ev = np.linalg.eigvalsh(A.toarray())
    b = rhs_uniform(A.shape[0], 1, config=97)[0]
    t, al, be = solvers.cg_sample(A, b, 40)
    kap = solvers.lanczos_condition_estimate(al, be)
    true = ev[-1] / ev[0]
    assert kap <= true * (1 + 1e-8)
    assert kap >= 0.9 * true
