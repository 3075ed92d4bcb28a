"""Pins of the oracle's grid and finite-volume assembly (CPU only).

Each test checks the oracle against something other than itself: the
calculus of the tanh map, the closed-form spectrum of the uniform Dirichlet
Laplacian, the exact flux of a piecewise-linear profile, and the Kronecker
structure of a separable problem.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fv, grid, solvers


# ---------------------------------------------------------------- grid (eq. "tanh")

@pytest.mark.parametrize("N", [8, 64, 256])
def test_tanh_nodes_endpoints_symmetry(N):
    x = grid.nodes_1d(N, 1.5)
    assert x[0] == 0.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    h = np.diff(x)
    hw = grid.widths_1d(N, 1.5)
    # widths of mirror cells equal bit for bit
    assert np.array_equal(hw, hw[::-1])
    assert np.allclose(h, hw, rtol=1e-12, atol=0)
    assert abs(hw.sum() - 1.0) < 1e-14


def test_tanh_wall_clustering_matches_derivative():
    # dx/di is proportional to sech^2(gamma (2 i / N - 1)): the width ratio
    # between the wall cell and the mid cell tends to sech^2(gamma).
    gamma, N = 1.5, 4096
    h = grid.widths_1d(N, gamma)
    ratio = h[0] / h[N // 2 - 1]
    sech2 = lambda z: 1.0 / np.cosh(z) ** 2
    zc_wall = gamma * (2 * 0.5 / N - 1)
    zc_mid = gamma * (2 * (N / 2 - 0.5) / N - 1)
    assert abs(ratio - sech2(zc_wall) / sech2(zc_mid)) < 1e-6
    assert abs(ratio - sech2(gamma)) < 2e-3


def test_tanh_uniform_limit():
    N = 32
    h = grid.widths_1d(N, 1e-7)
    assert np.max(np.abs(h - 1.0 / N)) < 1e-12


# ---------------------------------------------------------------- assembly

@pytest.mark.parametrize("N", [(6, 4), (5, 7), (4, 3, 5), (2, 6, 3)])
def test_uniform_spectrum_closed_form(N):
    h, k, A = fv.grid_operator(N, 0.0)
    ev = np.linalg.eigvalsh(A.toarray())
    cf = solvers.closed_form_eigenvalues(N)
    assert np.max(np.abs(ev - cf)) <= 1e-12 * cf.max()


def test_1d_variable_k_exact_flux_profile():
    # A piecewise-linear profile carrying a constant flux F through the
    # half-cell resistances h/(2k) is reproduced exactly by two-point fluxes:
    # (A u)_i = 0 for every cell but the last, whose high boundary face
    # carries F + t_high u_{N-1} out of the domain.
    rng = np.random.default_rng(3)
    n = 17
    hx = rng.uniform(0.2, 1.5, n)
    k = np.exp(rng.standard_normal(n))
    F = 0.7
    half = hx / (2 * k)
    u = np.empty(n)
    u[0] = F * half[0]
    for i in range(1, n):
        u[i] = u[i - 1] + F * (half[i - 1] + half[i])
    A = fv.assemble([hx], k)
    Au = A @ u
    assert np.max(np.abs(Au[:-1])) < 1e-12 * np.max(np.abs(u))
    t_high = 1.0 / half[-1]
    assert abs(Au[-1] - (F + t_high * u[-1])) < 1e-12 * abs(Au[-1])


def _kron3(Z, Y, X):
    return sp.kron(sp.kron(Z, Y), X)


def test_3d_separable_kronecker_structure():
    # k = k(x) only: A = Hz (x) Hy (x) Tx[k] + Hz (x) Ty (x) Dx + Tz (x) Hy (x) Dx
    # with T the 1D operators, H = diag(widths), Dx = diag(hx * k).
    rng = np.random.default_rng(5)
    N = (5, 4, 3)
    h = [rng.uniform(0.3, 1.2, n) for n in N]
    kx = np.exp(rng.standard_normal(N[0]))
    k3 = np.broadcast_to(kx[None, None, :], N[::-1]).reshape(-1)
    A = fv.assemble(h, k3).toarray()
    Tx = fv.assemble([h[0]], kx)
    Ty = fv.assemble([h[1]], np.ones(N[1]))
    Tz = fv.assemble([h[2]], np.ones(N[2]))
    Hy, Hz = sp.diags(h[1]), sp.diags(h[2])
    Dx = sp.diags(h[0] * kx)
    B = (_kron3(Hz, Hy, Tx) + _kron3(Hz, Ty, Dx) + _kron3(Tz, Hy, Dx)).toarray()
    assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(B))


def test_3d_separable_kronecker_structure_k_along_z():
    rng = np.random.default_rng(6)
    N = (3, 4, 5)
    h = [rng.uniform(0.3, 1.2, n) for n in N]
    kz = np.exp(rng.standard_normal(N[2]))
    k3 = np.broadcast_to(kz[:, None, None], N[::-1]).reshape(-1)
    A = fv.assemble(h, k3).toarray()
    Tz = fv.assemble([h[2]], kz)
    Tx = fv.assemble([h[0]], np.ones(N[0]))
    Ty = fv.assemble([h[1]], np.ones(N[1]))
    Hx, Hy = sp.diags(h[0]), sp.diags(h[1])
    Dz = sp.diags(h[2] * kz)
    B = (_kron3(Tz, Hy, Hx) + _kron3(Dz, Ty, Hx) + _kron3(Dz, Hy, Tx)).toarray()
    assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(B))


def test_assembly_symmetric_spd_and_matrix_free_apply():
    from synth import gaussian_logk

    N = (8, 6, 4)
    g = gaussian_logk(N, 1, seed=11, corr=2.0)
    h, k, A = fv.grid_operator(N, 1.5, g)
    Ad = A.toarray()
    assert np.array_equal(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad).min() > 0
    # off-diagonals non-positive, interior rows sum to zero
    off = Ad - np.diag(np.diag(Ad))
    assert off.max() <= 0
    u = np.random.default_rng(0).standard_normal(A.shape[0])
    assert np.max(np.abs(fv.apply(h, k, u) - A @ u)) < 1e-12 * np.max(np.abs(A @ u))
    # 7-point pattern: at most 7 entries per row
    assert np.diff(A.indptr).max() == 7
