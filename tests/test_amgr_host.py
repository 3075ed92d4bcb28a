"""AMGR setup on the host (Sec. 3.2; CPU only): the populated coarsening of
Alg. "popul", the prolongation of eq. "amgreduction" and the reduced operator
of eq. "structAc", checked against their definitions with the oracle's
operator.

* every interface point (a base row coupled to another mirror copy) is
  coarse; the selected inner points are independent at distance k in the
  strength graph of the inner points, and maximal (every inner fine point
  lies within distance k of one);
* P_b = [W; I]: a unit row per coarse point, and the fine rows of a
  zero-row-sum row of A_inn interpolate constants exactly;
* A_c = P^T A P with P = I (x) P_b, computed from the full unreduced
  operator in the mirrored order, equals the library's A_c.
"""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import paper_2407_05930_gb300 as amg
from oracle import fv, grid, symmetry
from synth import gaussian_logk


def _strength(A, theta=0.25):
    """Classical strength of connection by its definition: j strong for i
    when -a_ij >= theta * max_{k != i} (-a_ik)."""
    A = A.tocsr()
    rows, cols = [], []
    for i in range(A.shape[0]):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        c, v = A.indices[lo:hi], A.data[lo:hi]
        off = c != i
        if not np.any(off):
            continue
        mx = np.max(-v[off])
        if mx <= 0:
            continue
        for j, a in zip(c[off], v[off]):
            if -a >= theta * mx:
                rows.append(i)
                cols.append(j)
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=A.shape)


@pytest.mark.parametrize("N,s,bc,k", [((16, 12, 10), 1, "dirichlet", 1), ((12, 12, 8), 2, "neumann", 1),
                                      ((16, 12, 10), 1, "dirichlet", 2), ((12, 12, 8), 2, "neumann", 2),
                                      ((12, 8, 8), 3, "dirichlet", 2), ((14, 10, 8), 1, "dirichlet", 3)])
def test_populated_coarsening_prolongation_and_reduced_operator(N, s, bc, k):
    g = gaussian_logk(N, s, seed=31, corr=2.0)
    A = fv.assemble(grid.widths(N, 1.5), np.exp(g), bc)
    perm = symmetry.mirror_perm(N, s)
    P = amg.Problem(A.shape[0], A.indptr, A.indices, A.data, s, perm)
    P.setup(host_only=1, amgr=1, amgr_distance=k, coarse_max=64)
    info = P.amgr_info()
    cf = info["cf"]
    H = symmetry.blocks(A, perm)
    Ainn = H[0].tocsr()
    nb = 1 << s
    # interface: rows of the base block coupled to another copy
    iface = np.zeros(Ainn.shape[0], bool)
    for m in range(1, nb):
        iface |= np.diff(H[m].tocsr().indptr) > 0
    assert np.all(cf[iface] == 1)
    inner = ~iface
    # the strength graph of the inner points, symmetrised, and distances in it
    S = _strength(Ainn)
    T = ((S + S.T) > 0).astype(float)
    T = T[inner][:, inner]
    D = shortest_path(T, unweighted=True, directed=False)
    sel = cf[inner] == 1
    Dsel = D[np.ix_(sel, sel)]
    np.fill_diagonal(Dsel, np.inf)
    assert np.all(Dsel > k)  # independent at distance k
    assert np.all(np.min(D[:, sel], axis=1)[~sel] <= k)  # maximal
    # P_b = [W; I]
    rp, ci, v, shape = P.amgr_matrix("P")
    Pb = sp.csr_matrix((v, ci, rp), shape=shape)
    assert shape == (Ainn.shape[0], info["n_cb"]) and info["n_cb"] == int(np.sum(cf == 1))
    cidx = np.cumsum(cf == 1) - 1
    for i in np.flatnonzero(cf == 1):
        row = Pb.getrow(i)
        assert row.nnz == 1 and row.indices[0] == cidx[i] and row.data[0] == 1.0
    rowsum = np.asarray(Ainn.sum(axis=1)).ravel()
    diag = Ainn.diagonal()
    zero = (np.abs(rowsum) <= 1e-12 * diag) & (cf == -1) & (np.diff(Pb.indptr) > 0)
    assert np.any(zero)
    assert np.max(np.abs(np.asarray(Pb[zero].sum(axis=1)).ravel() - 1.0)) <= 1e-12
    # A_c = P^T A P in the interleaved mirrored order (base point l, copy j -> l * nb + j)
    n_b = Ainn.shape[0]
    order = np.empty(A.shape[0], dtype=np.int64)
    for j in range(nb):
        order[np.arange(n_b) * nb + j] = perm[j]
    Am = A[order][:, order]
    Pfull = sp.kron(Pb, sp.identity(nb), format="csr")
    Ac_ref = (Pfull.T @ Am @ Pfull).tocsr()
    rp, ci, v, shape = P.amgr_matrix("Ac")
    Ac = sp.csr_matrix((v, ci, rp), shape=shape)
    assert shape == Ac_ref.shape
    assert abs(Ac - Ac_ref).max() <= 1e-12 * abs(Ac_ref).max()
    assert info["levels"] >= 1


@pytest.mark.parametrize("N,s,bc", [((12, 12, 8), 2, "neumann"), ((12, 8, 8), 3, "dirichlet"),
                                    ((16, 12, 10), 1, "dirichlet")])
def test_reduced_operator_is_block_diagonal_in_the_transformed_basis(N, s, bc):
    """The identity behind the transformed-basis products of A_c (opts.amgr_sym_ac):
    with P = I (x) P_b commuting with P_s, block (p, q) of A_c (copies p, q) is
    2^-s sum_i s(i, p) s(i, q) A^_c,i with A^_c,i = P_b^T A^_i P_b (eq. "structAc"
    under eq. "P_s"), and A^_c,i - P_b^T A_inn P_b is the fine interface coupling
    A^_i - A_inn itself on the coarse indices of the interface points (they are
    coarse, with unit rows in P_b)."""
    from oracle import transform

    g = gaussian_logk(N, s, seed=33, corr=2.0)
    A = fv.assemble(grid.widths(N, 1.5), np.exp(g), bc)
    perm = symmetry.mirror_perm(N, s)
    P = amg.Problem(A.shape[0], A.indptr, A.indices, A.data, s, perm)
    P.setup(host_only=1, amgr=1, coarse_max=64)
    nb = 1 << s
    H = symmetry.blocks(A, perm)
    hat = transform.hat_blocks_sparse(H)
    rp, ci, v, shape = P.amgr_matrix("P")
    Pb = sp.csr_matrix((v, ci, rp), shape=shape)
    rp, ci, v, shape = P.amgr_matrix("Ac")
    Ac = sp.csr_matrix((v, ci, rp), shape=shape)
    hat_c = [(Pb.T @ Ai @ Pb).tocsr() for Ai in hat]
    scale = max(abs(Ac).max(), 1.0)
    for p in range(nb):
        for q in range(nb):
            blk = Ac[p::nb][:, q::nb]
            ref = sp.csr_matrix(blk.shape)
            for i in range(nb):
                ref = ref + transform.hadamard_sign(i, p) * transform.hadamard_sign(i, q) * hat_c[i]
            ref = ref / nb
            assert abs(blk - ref).max() <= 1e-12 * scale, (p, q)
    # the couplings of the transformed blocks are the fine ones at coarse indices
    cf = P.amgr_info()["cf"]
    cidx = np.cumsum(cf == 1) - 1
    inn_c = (Pb.T @ H[0] @ Pb).tocsr()
    for i in range(nb):
        fine = (hat[i] - H[0]).tocoo()
        if fine.nnz:
            assert np.all(cf[fine.row] == 1) and np.all(cf[fine.col] == 1)
        ref = sp.csr_matrix((fine.data, (cidx[fine.row], cidx[fine.col])), shape=inn_c.shape)
        assert abs((hat_c[i] - inn_c) - ref).max() <= 1e-12 * scale, i
