"""Host-side logic of the C ABI (CPU only, no CUDA call).

* every symbol declared in include/amgsym.h is exported by libamgsym.so;
* the library's structured-grid generator and mirror map agree with the
  oracle (map bit-exact, matrix to rounding);
* create_problem validates the map and the block structure of eq.
  "struct_2sym", and extracts A_inn and A_out,i equal to the oracle's blocks;
* the AMG hierarchy has the structure the V-cycle relies on.
"""

import ctypes
import re

import numpy as np
import pytest
import scipy.sparse as sp

import paper_2407_05930_gb300 as amg
from oracle import fv, grid, symmetry, transform
from synth import gaussian_logk

import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_symbols_exported():
    hdr = open(os.path.join(ROOT, "include", "amgsym.h")).read()
    names = set(re.findall(r"\b(amgsym_[a-z_0-9]+)\s*\(", hdr))
    assert names, "no declarations found"
    lib = ctypes.CDLL(amg.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(amg.EXPORTED) <= names


@pytest.mark.parametrize("N,gamma", [((64,), 0.0), ((10, 8), 1.5), ((6, 8, 4), 1.5), ((256,), 1.5)])
def test_generator_matches_oracle(N, gamma):
    w = [amg.grid_widths(n, gamma) for n in N]
    h = grid.widths(N, gamma)
    for a, b in zip(w, h):
        assert np.max(np.abs(a - b)) <= 4e-16
        if a.size % 2 == 0:
            assert np.array_equal(a, a[::-1])
    rng = np.random.default_rng(0)
    k = np.exp(rng.standard_normal(int(np.prod(N))))
    rp, ci, v = amg.fv_assemble(N, w, k)
    Ap = sp.csr_matrix((v, ci, rp), shape=(k.size, k.size))
    Ao = fv.assemble(h, k)
    assert (Ap != 0).nnz == Ao.nnz
    # entrywise relative agreement: the widths are differences of nodes near
    # 1/2, so one ulp of tanh becomes ~1e-13 relative in a wall-cell width
    D = (Ap - Ao).tocoo()
    ref = np.asarray(abs(Ao)[D.row, D.col]).ravel()
    assert np.all(np.abs(D.data) <= 1e-12 * ref)


@pytest.mark.parametrize("N,s", [((8, 6), 1), ((8, 8), 2), ((6, 4, 8), 3), ((4, 6, 2), 2), ((10,), 1), ((6, 4, 4), 0)])
def test_mirror_perm_bit_exact(N, s):
    assert np.array_equal(amg.mirror_perm(N, s), symmetry.mirror_perm(N, s))


def _oracle_problem(N, s, gamma=1.5, seed=2):
    g = gaussian_logk(N, s, seed=seed, corr=1.5)
    h, k, A = fv.grid_operator(N, gamma, g)
    return g, A


@pytest.mark.parametrize("N,s", [((8, 6), 1), ((6, 8, 4), 3), ((8, 4, 6), 2)])
def test_create_problem_extracts_oracle_blocks(N, s):
    g, A = _oracle_problem(N, s)
    perm = symmetry.mirror_perm(N, s)
    P = amg.Problem(A.shape[0], A.indptr, A.indices, A.data, s, perm)
    rp, ci, v = P.inner_block()
    Ainn = sp.csr_matrix((v, ci, rp), shape=(P.n_b, P.n_b))
    H = symmetry.blocks(A, perm)
    assert (Ainn != H[0]).nnz == 0  # bit-exact extraction
    r, c, iv = P.interface()
    hat = transform.hat_blocks_sparse(H)
    for i in range(1 << s):
        Aout = sp.csr_matrix((iv[:, i], (r, c)), shape=Ainn.shape)
        ref = hat[i] - H[0]
        assert abs(Aout - ref).max() <= 1e-15 * abs(H[0]).max()


def test_create_problem_rejects_bad_map():
    g, A = _oracle_problem((8, 6), 1)
    perm = symmetry.mirror_perm((8, 6), 1).copy()
    perm[1, 0] = perm[0, 0]
    with pytest.raises(amg.AmgsymError) as e:
        amg.Problem(A.shape[0], A.indptr, A.indices, A.data, 1, perm)
    assert e.value.name == "ERR_MAP"
    perm = symmetry.mirror_perm((8, 6), 1).copy()
    perm[0, 0] = 10**6
    with pytest.raises(amg.AmgsymError) as e:
        amg.Problem(A.shape[0], A.indptr, A.indices, A.data, 1, perm)
    assert e.value.name == "ERR_MAP"


def test_create_problem_rejects_asymmetric_coefficient():
    N = (8, 6)
    g = np.random.default_rng(1).standard_normal(48)  # breaks the mirror symmetry
    h, k, A = fv.grid_operator(N, 0.0, g)
    perm = symmetry.mirror_perm(N, 1)
    with pytest.raises(amg.AmgsymError) as e:
        amg.Problem(A.shape[0], A.indptr, A.indices, A.data, 1, perm)
    assert e.value.name == "ERR_NOT_SYMMETRIC"


def test_create_problem_rejects_nonsymmetric_matrix():
    g, A = _oracle_problem((8, 6), 1)
    A = A.tolil()
    # perturb one pair of mirror entries consistently but not symmetrically
    perm = symmetry.mirror_perm((8, 6), 1)
    p0, q0 = perm[0, 0], perm[0, 1]
    p1, q1 = perm[1, 0], perm[1, 1]
    A[p0, q0] = A[p0, q0] * 1.5
    A[p1, q1] = A[p1, q1] * 1.5
    A = A.tocsr()
    with pytest.raises(amg.AmgsymError) as e:
        amg.Problem(A.shape[0], A.indptr, A.indices, A.data, 1, perm)
    assert e.value.name == "ERR_NOT_SYMMETRIC"


def test_create_problem_rejects_bad_csr():
    g, A = _oracle_problem((8, 6), 1)
    perm = symmetry.mirror_perm((8, 6), 1)
    ci = A.indices.copy()
    ci[3] = -1
    with pytest.raises(amg.AmgsymError) as e:
        amg.Problem(A.shape[0], A.indptr, ci, A.data, 1, perm)
    assert e.value.name == "ERR_ARG"
    with pytest.raises(amg.AmgsymError):
        amg.Problem(A.shape[0], A.indptr, A.indices, A.data, 1, perm[:, :-1].copy().reshape(-1)[: A.shape[0] - 2])


def _csr(t):
    rp, ci, v, shape = t
    return sp.csr_matrix((v, ci, rp), shape=shape)


@pytest.mark.parametrize("drop", [0.0, 0.01])
def test_hierarchy_structure(drop):
    N, s = (32, 32, 32), 3
    g = gaussian_logk(N, s, seed=3, corr=4.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, coarse_max=128, coarse_drop=drop)
    L = P.num_levels()
    assert L >= 3
    A0 = _csr(P.level_matrix(0, "A"))
    rp, ci, v = P.inner_block()
    assert (A0 != sp.csr_matrix((v, ci, rp), shape=A0.shape)).nnz == 0
    for l in range(L - 1):
        A = _csr(P.level_matrix(l, "A"))
        Pm = _csr(P.level_matrix(l, "P"))
        G = _csr(P.level_matrix(l, "G"))
        Ac = _csr(P.level_matrix(l + 1, "A"))
        # Galerkin coarse operator R A P with R = P^T; sparsified: small
        # couplings moved to the diagonal (row sums and symmetry kept)
        ref = (Pm.T @ A @ Pm).tocsr()
        # symmetrised exactly: each pair (i, j), (j, i) holds one value
        assert (Ac != Ac.T).nnz == 0
        if drop == 0.0:
            assert abs(Ac - ref).max() <= 1e-12 * abs(ref).max()
        else:
            one = np.ones(ref.shape[0])
            assert np.max(np.abs(Ac @ one - ref @ one)) <= 1e-12 * abs(ref).max()
            assert abs(Ac - Ac.T).max() <= 1e-12 * abs(ref).max()
            d = Ac.diagonal()
            off = (Ac - sp.diags(d)).tocoo()
            assert np.all(np.abs(off.data) >= drop * np.sqrt(d[off.row] * d[off.col]) * (1 - 1e-12))
            assert Ac.nnz <= ref.nnz
        # C points interpolate by injection: some rows are unit vectors
        assert np.isclose(Pm.max(), 1.0) or Pm.max() >= 1.0
        # FSAI: lower triangular, G A G^T has unit diagonal
        assert sp.triu(G, k=1).nnz == 0
        d = (G @ A @ G.T).diagonal()
        assert np.max(np.abs(d - 1.0)) < 1e-10
        inf = P.level_info(l)
        assert 0.0 < inf["omega"] < 2.0
    assert P.level_info(L - 1)["rows"] <= 128


@pytest.mark.parametrize("N,s", [((12, 10, 8), 3), ((64, 64), 1), ((10, 8, 6), 0)])
def test_diagonal_form_detection(N, s):
    """The diagonal-offset copies of the structured-grid operators: the base
    block of a d-dimensional stencil has the 2d+1 offsets 0, +-1, +-nx,
    +-nx*ny (x fastest), stores its lower half only (exactly symmetric
    finite-volume matrix); its FSAI factor G has the lower offsets and G^T
    the upper ones, all stored; no diagonal form above AMGSYM_MAX_DIAG or
    with dia_max_diag = 0."""
    g = gaussian_logk(N, s, seed=4, corr=2.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, coarse_max=32)
    base = list(N)
    for a in range(s):
        base[a] //= 2
    strides = [int(np.prod(base[:a])) for a in range(len(base))]
    lower = sorted([-t for t in strides] + [0])
    full = sorted(set(lower + [t for t in strides]))
    A = P.level_dia(0, "A")
    assert A["offsets"] == full and A["ndiag"] == 2 * len(N) + 1
    assert A["nstored"] == len(N) + 1
    G, Gt = P.level_dia(0, "G"), P.level_dia(0, "Gt")
    assert G["offsets"] == lower and G["nstored"] == G["ndiag"]
    assert Gt["offsets"] == sorted(-o for o in lower) and Gt["nstored"] == Gt["ndiag"]
    # the stored diagonal form reproduces the CSR matrix: checked on the GPU
    # (bit-identical products); here its pattern must cover every entry
    rp, ci, v, shape = P.level_matrix(0, "A")
    rows = np.repeat(np.arange(shape[0]), np.diff(rp))
    assert set(np.unique(ci - rows).tolist()) <= set(full)
    Q = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, coarse_max=32, dia_max_diag=0)
    assert Q.level_dia(0, "A")["ndiag"] == 0 and Q.level_dia(0, "G")["ndiag"] == 0
    R = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, coarse_max=32, dia_max_diag=len(N) * 2)
    assert R.level_dia(0, "A")["ndiag"] == 0 and R.level_dia(0, "G")["ndiag"] == len(N) + 1
    assert amg.lib.amgsym_level_dia(P._h, 0, 1, None, None, None) == -1  # P has no diagonal form
    with pytest.raises(amg.AmgsymError):
        P.level_dia(P.num_levels(), "A")


def test_coarse_levels_take_a_diagonal_fsai_factor():
    """fsai_max_lower_coarse: the finest level keeps the 4-entry lower FSAI
    pattern of a 7-point stencil, every coarse level a diagonal one (damped
    Jacobi with the same omega rule); with 4 the coarse factors are not
    diagonal.  A diagonal G is D^{-1/2}-like: positive, so G^T G is SPD."""
    N, s = (24, 20, 16), 2
    g = gaussian_logk(N, s, seed=6, corr=2.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, coarse_max=32)
    assert P.num_levels() >= 3
    rp, ci, v, shape = P.level_matrix(0, "G")
    assert np.max(np.diff(rp)) == 4
    for l in range(1, P.num_levels() - 1):
        rp, ci, v, shape = P.level_matrix(l, "G")
        rows = np.arange(shape[0])
        assert np.array_equal(np.diff(rp), np.ones(shape[0], dtype=np.int64))
        assert np.array_equal(ci, rows) and np.all(v > 0)
    Q = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, coarse_max=32, fsai_max_lower_coarse=4)
    rp, ci, v, shape = Q.level_matrix(1, "G")
    assert np.max(np.diff(rp)) > 1
    with pytest.raises(amg.AmgsymError):
        amg.Problem.structured(N, 1.5, g, s).setup(host_only=1, fsai_max_lower_coarse=0)


@pytest.mark.parametrize("N,s", [((8, 6, 4), 3), ((10, 6), 1)])
def test_update_values_replaces_blocks_and_rejects_broken_symmetry(N, s):
    """amgsym_update_values: a new coefficient field on the same pattern gives
    exactly the oracle's blocks of the new operator; values that break the
    block structure are rejected and leave the problem as it was; an
    accepted update drops the hierarchy until the next setup."""
    h = grid.widths(N, 1.5)
    perm = symmetry.mirror_perm(N, s)
    g1 = gaussian_logk(N, s, seed=8, corr=2.0)
    g2 = gaussian_logk(N, s, seed=9, corr=2.0)
    A1 = fv.assemble(h, np.exp(g1))
    A2 = fv.assemble(h, np.exp(g2))
    assert np.array_equal(A1.indptr, A2.indptr) and np.array_equal(A1.indices, A2.indices)
    P = amg.Problem(A1.shape[0], A1.indptr, A1.indices, A1.data, s, perm)
    P.setup(host_only=1, coarse_max=16)
    assert P.num_levels() >= 2
    P.update_values(A2.data)
    assert P.num_levels() == 0  # hierarchy released
    rp, ci, v = P.inner_block()
    Ainn = sp.csr_matrix((v, ci, rp), shape=(P.n_b, P.n_b))
    H = symmetry.blocks(A2, perm)
    assert (Ainn != H[0]).nnz == 0
    r, c, iv = P.interface()
    hat = transform.hat_blocks_sparse(H)
    for i in range(1 << s):
        Aout = sp.csr_matrix((iv[:, i], (r, c)), shape=Ainn.shape)
        assert abs(Aout - (hat[i] - H[0])).max() <= 1e-15 * abs(H[0]).max()
    # one entry of one mirror copy changed: rejected, nothing modified
    bad = A1.data.copy()
    p = perm[1, 5] if s > 0 else 5
    bad[A1.indptr[p]] *= 1.5
    with pytest.raises(amg.AmgsymError) as e:
        P.update_values(bad)
    assert e.value.name == "ERR_NOT_SYMMETRIC"
    rp2, ci2, v2 = P.inner_block()
    assert np.array_equal(v2, v) and np.array_equal(ci2, ci)
    P.setup(host_only=1, coarse_max=16)
    assert P.num_levels() >= 2


@pytest.mark.parametrize("name", ["zmarch", "sell", "amgr_sym_ac", "lambda_device"])
def test_kernel_form_options_are_validated(name):
    """The kernel-form switches (z-marching stencil, sliced CSR, AMGR coarse
    operator in the transformed basis) take 0 or 1; their defaults are
    reported by amgsym_opts_default."""
    o = amg.default_opts()
    assert getattr(o, name) in (0, 1)
    assert (o.zmarch, o.sell, o.amgr_sym_ac, o.lambda_device) == (0, 0, 1, 1)
    P = amg.Problem.structured((8, 8, 8), 0.0, None, 1)
    with pytest.raises(amg.AmgsymError) as e:
        P.setup(host_only=1, **{name: 2})
    assert e.value.name == "ERR_ARG"
    P.setup(host_only=1, **{name: 1})
    assert P.num_levels() >= 1
