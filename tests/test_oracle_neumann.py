"""Pins of the oracle's Neumann model problem (Sec. 2.2, eq. "modelproblem":
homogeneous Neumann on every wall of the unit cube), and of the library's
host-side handling of it (generator, singularity detection, setup).

* the assembled operator is symmetric, every row sums to zero, and on a
  uniform grid its spectrum is the closed form sum_a c_a 4 sin^2(m_a pi /
  (2 N_a)) with m_a = 0..N_a-1 (one zero eigenvalue);
* the cosine-transform solve, the dense minimum-norm solve and plain CG on
  the consistent singular system give the same zero-mean solution;
* the symmetry split still holds: the block spectra union equals the full
  spectrum; only the all-"+" block A^_0 is singular, A_inn is regular (s >= 1).
"""

import numpy as np
import pytest
import scipy.sparse as sp

import paper_2407_05930_gb300 as amg
from oracle import fv, grid, solvers, symmetry, transform
from synth import gaussian_logk


@pytest.mark.parametrize("N", [(7, 5, 4), (9, 6), (12,)])
def test_neumann_operator_closed_form(N):
    h = grid.widths(N, 0.0)
    n = int(np.prod(N))
    A = fv.assemble(h, np.ones(n), "neumann")
    Ad = A.toarray()
    assert np.array_equal(Ad, Ad.T)
    assert np.max(np.abs(Ad.sum(axis=1))) <= 1e-14 * np.max(np.abs(Ad))
    ev = np.linalg.eigvalsh(Ad)
    cf = solvers.closed_form_eigenvalues(N, "neumann")
    assert np.max(np.abs(ev - cf)) <= 1e-12 * cf[-1]
    assert abs(cf[0]) == 0.0 and cf[1] > 0.0
    # Dirichlet differs only on the wall rows: the wall transmissibility
    D = fv.assemble(h, np.ones(n)) - A
    assert np.all(D.diagonal() >= 0) and (D - sp.diags(D.diagonal())).nnz == 0


def test_neumann_matrix_free_apply_equals_assembly():
    N = (8, 6, 4)
    h = grid.widths(N, 1.5)
    k = np.exp(gaussian_logk(N, 1, seed=2, corr=2.0))
    A = fv.assemble(h, k, "neumann")
    u = np.random.default_rng(1).standard_normal(A.shape[0])
    assert np.linalg.norm(fv.apply(h, k, u, "neumann") - A @ u) <= 1e-13 * np.linalg.norm(A @ u)
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) <= 1e-14 * abs(A).max()


def test_three_solvers_agree_on_the_minimum_norm_solution():
    N = (10, 8, 6)
    h = grid.widths(N, 0.0)
    A = fv.assemble(h, np.ones(int(np.prod(N))), "neumann")
    b = np.random.default_rng(3).uniform(-1, 1, (2, A.shape[0]))
    b -= b.mean(axis=1, keepdims=True)  # compatibility: 1^T b = 0
    x_dct = solvers.neumann_dct_solve(N, b)
    for r in range(2):
        x_min = solvers.min_norm_solve(A, b[r])
        x_cg = solvers.cg(A, b[r], tol=1e-13)
        x_cg -= x_cg.mean()
        assert abs(x_dct[r].mean()) <= 1e-14 * np.abs(x_dct[r]).max()
        assert np.linalg.norm(x_dct[r] - x_min) <= 1e-11 * np.linalg.norm(x_min)
        assert np.linalg.norm(x_cg - x_min) <= 1e-10 * np.linalg.norm(x_min)
        assert np.linalg.norm(A @ x_dct[r] - b[r]) <= 1e-12 * np.linalg.norm(b[r])


@pytest.mark.parametrize("N,s", [((8, 6, 4), 1), ((8, 6, 4), 2), ((6, 4, 8), 3)])
def test_neumann_blocks(N, s):
    h = grid.widths(N, 1.5)
    k = np.exp(gaussian_logk(N, s, seed=4, corr=2.0))
    A = fv.assemble(h, k, "neumann")
    perm = symmetry.mirror_perm(N, s)
    H = symmetry.blocks(A, perm)
    hat = transform.hat_blocks_sparse(H)
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(Hi.toarray()) for Hi in hat]))
    full = np.linalg.eigvalsh(A.toarray())
    assert np.max(np.abs(ev - full)) <= 1e-12 * full[-1]
    lam0 = np.linalg.eigvalsh(hat[0].toarray())
    assert abs(lam0[0]) <= 1e-12 * lam0[-1]  # the symmetric mode keeps the constant
    for Hi in hat[1:]:
        assert np.linalg.eigvalsh(Hi.toarray())[0] > 1e-8 * full[-1]
    assert np.linalg.eigvalsh(H[0].toarray())[0] > 1e-8 * full[-1]  # A_inn regular


@pytest.mark.parametrize("N,gamma", [((10, 8), 1.5), ((6, 8, 4), 1.5)])
def test_library_generator_and_singularity(N, gamma):
    w = [amg.grid_widths(n, gamma) for n in N]
    h = grid.widths(N, gamma)
    k = np.exp(np.random.default_rng(0).standard_normal(int(np.prod(N))))
    rp, ci, v = amg.fv_assemble(N, w, k, "neumann")
    Ap = sp.csr_matrix((v, ci, rp), shape=(k.size, k.size))
    Ao = fv.assemble(h, k, "neumann")
    D = (Ap - Ao).tocoo()
    ref = np.asarray(abs(Ao)[D.row, D.col]).ravel()
    assert np.all(np.abs(D.data) <= 1e-12 * ref)
    kk = np.exp(gaussian_logk(N, 1, seed=3, corr=2.0))
    for s in (0, 1):
        Pn = amg.Problem.structured(N, gamma, np.log(kk), s, bc="neumann")
        Pd = amg.Problem.structured(N, gamma, np.log(kk), s)
        assert Pn.singular and not Pd.singular
        # host setup: with s = 0 the hierarchy is of the singular operator
        # itself and its coarsest level takes the pseudo-inverse
        Pn.setup(host_only=1, coarse_max=16)
        assert Pn.num_levels() >= 2
