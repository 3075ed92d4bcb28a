"""Pins of the oracle's mirrored ordering, ``P_s`` and decoupled blocks (CPU only).

Against: brute-force loops, the exact algebra of eqs. "P_s", "hL_s1", "hL_s"
(orthonormality, involution, block diagonalisation, spectrum union), the
closed-form 1D split spectra and energy placement of (anti)symmetric inputs.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fv, solvers, symmetry, transform
from synth import gaussian_logk

CASES = [((8, 6), 1), ((8, 8), 2), ((4, 6, 4), 3), ((6, 4, 2), 2), ((10,), 1)]


def _problem(N, s, gamma=1.5, seed=1):
    logk = gaussian_logk(N, s, seed=seed, corr=1.5) if len(N) > 1 else None
    if logk is None:
        logk = np.zeros(N[0])
    h, k, A = fv.grid_operator(N, gamma, logk)
    return h, k, A


@pytest.mark.parametrize("N,s", CASES)
def test_perm_bijection_and_bruteforce(N, s):
    perm = symmetry.mirror_perm(N, s)
    assert np.array_equal(perm, symmetry.mirror_perm_bruteforce(N, s))
    n = int(np.prod(N))
    assert np.array_equal(np.sort(perm.reshape(-1)), np.arange(n))
    # copy 0 is the all-lower octant
    M = symmetry.base_shape(N, s)
    coords = np.unravel_index(perm[0], N[::-1])[::-1]
    for b in range(s):
        assert coords[b].max() < M[b]


@pytest.mark.parametrize("N,s", CASES)
def test_dyadic_block_structure_exact(N, s):
    h, k, A = _problem(N, s)
    perm = symmetry.mirror_perm(N, s)
    assert symmetry.check_dyadic_structure(A, perm) == 0.0


def test_dyadic_structure_detects_asymmetric_coefficient():
    N, s = (8, 6), 1
    g = np.random.default_rng(2).standard_normal(48)  # not mirror symmetric
    h, k, A = fv.grid_operator(N, 0.0, g)
    perm = symmetry.mirror_perm(N, s)
    assert symmetry.check_dyadic_structure(A, perm) > 1e-3


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_P_s_orthonormal_involution(s):
    n = 8 * 3
    P = transform.P_s_dense(s, n)
    assert np.allclose(P @ P, np.eye(n), atol=1e-14)
    assert np.allclose(P, P.T, atol=0)
    x = np.random.default_rng(s).standard_normal((3, n))
    assert np.allclose(transform.P_s_apply(s, x), x @ P.T, atol=1e-14)


@pytest.mark.parametrize("N,s", CASES)
def test_block_diagonalisation_and_hat_blocks(N, s):
    h, k, A = _problem(N, s)
    perm = symmetry.mirror_perm(N, s)
    order = symmetry.mirror_order(perm)
    Am = A.toarray()[np.ix_(order, order)]
    blocks, off = transform.decoupled_blocks_dense(Am, s)
    scale = np.max(np.abs(Am))
    assert off <= 1e-13 * scale
    H = symmetry.blocks(A, perm)
    hat = transform.hat_blocks_sparse(H)
    for i in range(1 << s):
        assert np.max(np.abs(blocks[i] - hat[i].toarray())) <= 1e-13 * scale
    # union of the block spectra is the spectrum of A
    ev = np.sort(np.linalg.eigvalsh(Am))
    evb = np.sort(np.concatenate([np.linalg.eigvalsh(b) for b in blocks]))
    assert np.max(np.abs(ev - evb)) <= 1e-12 * ev.max()


def test_single_symmetry_closed_form_blocks():
    # eq. "hL_s1": P_1 A P_1^{-1} = diag(A_1 + A_2, A_1 - A_2)
    h, k, A = _problem((8, 6), 1)
    perm = symmetry.mirror_perm((8, 6), 1)
    order = symmetry.mirror_order(perm)
    Am = A.toarray()[np.ix_(order, order)]
    m = Am.shape[0] // 2
    A1, A2 = Am[:m, :m], Am[:m, m:]
    blocks, _ = transform.decoupled_blocks_dense(Am, 1)
    assert np.allclose(blocks[0], A1 + A2, atol=1e-13)
    assert np.allclose(blocks[1], A1 - A2, atol=1e-13)


def test_1d_split_spectra_odd_even_modes():
    N = 12
    h, k, A = fv.grid_operator((N,), 0.0)
    perm = symmetry.mirror_perm((N,), 1)
    order = symmetry.mirror_order(perm)
    blocks, _ = transform.decoupled_blocks_dense(A.toarray()[np.ix_(order, order)], 1)
    c = 1.0 / (1.0 / N)  # area 1 over width 1/N
    m = np.arange(1, N + 1)
    lam = c * 4 * np.sin(m * np.pi / (2 * N)) ** 2
    assert np.allclose(np.sort(np.linalg.eigvalsh(blocks[0])), np.sort(lam[m % 2 == 1]), rtol=1e-12)
    assert np.allclose(np.sort(np.linalg.eigvalsh(blocks[1])), np.sort(lam[m % 2 == 0]), rtol=1e-12)


def test_energy_placement_of_symmetric_inputs():
    N, s = (4, 6, 4), 3
    perm = symmetry.mirror_perm(N, s)
    n_b = perm.shape[1]
    base = np.random.default_rng(9).standard_normal(n_b)
    # fully symmetric: every copy equal -> only block 0
    xm = np.tile(base, 1 << s)
    y = transform.P_s_apply(s, xm).reshape(1 << s, n_b)
    assert np.max(np.abs(y[1:])) < 1e-14 and np.max(np.abs(y[0])) > 0.1
    # antisymmetric about plane b: copies with bit b set carry the sign
    for b in range(s):
        sign = np.array([-1.0 if (j >> b) & 1 else 1.0 for j in range(1 << s)])
        xm = (sign[:, None] * base[None, :]).reshape(-1)
        y = transform.P_s_apply(s, xm).reshape(1 << s, n_b)
        for i in range(1 << s):
            if (i >> b) & 1:
                continue
            assert np.max(np.abs(y[i])) < 1e-14


@pytest.mark.parametrize("N,s", [((8, 6), 1), ((4, 6, 4), 3), ((8, 8), 2)])
def test_reduced_solve_equals_full_solve(N, s):
    # Alg. 1: b^ = P_s b, solve each A^_i x^_i = b^_i, x = P_s x^.
    h, k, A = _problem(N, s)
    perm = symmetry.mirror_perm(N, s)
    order = symmetry.mirror_order(perm)
    b = np.random.default_rng(4).uniform(-1, 1, A.shape[0])
    x_full = solvers.dense_solve(A, b)
    H = symmetry.blocks(A, perm)
    hat = transform.hat_blocks_sparse(H)
    bh = transform.P_s_apply(s, b[order]).reshape(1 << s, -1)
    xh = np.stack([solvers.dense_solve(hat[i], bh[i]) for i in range(1 << s)])
    xm = transform.P_s_apply(s, xh.reshape(-1))
    x = np.empty_like(xm)
    x[order] = xm
    assert np.linalg.norm(x - x_full) <= 1e-12 * np.linalg.norm(x_full)


def test_interface_blocks_are_diagonal_for_7pt():
    h, k, A = _problem((4, 6, 4), 3)
    perm = symmetry.mirror_perm((4, 6, 4), 3)
    H = symmetry.blocks(A, perm)
    for j in range(1, 8):
        offd = H[j] - sp.diags(H[j].diagonal())
        if bin(j).count("1") == 1:
            assert abs(offd).max() == 0 if offd.nnz else True
            assert H[j].nnz > 0
        else:
            assert H[j].nnz == 0 or abs(H[j]).max() == 0
