"""AMGR (Sec. 3.2, Alg. "apply"; marked gpu): the multigrid reduction as the
preconditioner of the reduced PCG.

* the AMGR V-cycle is symmetric and positive definite (FP64, random vectors);
* PCG + AMGR solves the full system: parity with the oracle's exact solves
  (DST on uniform grids, sparse direct on stretched variable-coefficient
  ones), FP64 and mixed precision;
* the paper's model problem (Neumann, tanh 1.5, s = 0..3): AMGR converges in
  fewer iterations than I (x) M_inn^{-1}, as in Tables "lrcamg" and "amgr"
  (the counts themselves depend on the AMG and are not pinned).
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from oracle import fv, grid, solvers  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("s", [1, 3])
def test_amgr_vcycle_is_spd(s):
    N = (32, 24, 16)
    g = gaussian_logk(N, s, seed=33, corr=2.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(amgr=1, coarse_max=64)
    C = 2 << s
    rng = np.random.default_rng(4)
    U = torch.from_numpy(rng.standard_normal((P.n_b, C))).to(DEV)
    V = torch.from_numpy(rng.standard_normal((P.n_b, C))).to(DEV)
    MU, MV = torch.empty_like(U), torch.empty_like(V)
    P.amgr_apply(U, MU, 2, amg.PREC_FP64)
    P.amgr_apply(V, MV, 2, amg.PREC_FP64)
    # the AMG of A_c over the full coarse domain couples the blocks of one
    # right-hand side, so the operator is symmetric over each RHS's columns
    nb = 1 << s
    a = (MU * V).sum(dim=0).cpu().numpy().reshape(2, nb).sum(axis=1)
    b = (U * MV).sum(dim=0).cpu().numpy().reshape(2, nb).sum(axis=1)
    assert np.max(np.abs(a - b) / np.abs(a)) <= 1e-10
    assert np.all((MU * U).sum(dim=0).cpu().numpy().reshape(2, nb).sum(axis=1) > 0)


@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_amgr_pcg_uniform_matches_dst(s, prec):
    N = (32, 32, 32)
    P = amg.Problem.structured(N, 0.0, None, s).setup(amgr=1)
    b = rhs_uniform(P.n, 2, config=95)
    tol = 1e-12 if prec == amg.PREC_FP64 else 1e-10
    x, info = P.solve(torch.from_numpy(b).to(DEV), tol=tol, precision=prec, preconditioner=amg.PC_AMGR)
    assert info.converged and np.all(info.relres <= tol), info
    xo = solvers.dst_solve(N, b)
    xg = x.cpu().numpy()
    for r in range(2):
        assert _rel(xg[r], xo[r]) <= (1e-8 if prec == amg.PREC_FP64 else 1e-6)


def test_amgr_pcg_stretched_varcoef():
    N, s = (24, 20, 16), 2
    g = gaussian_logk(N, s, seed=96, corr=2.0)
    h, k, A = fv.grid_operator(N, 1.5, g)
    P = amg.Problem.structured(N, 1.5, g, s).setup(amgr=1, coarse_max=64)
    b = rhs_uniform(P.n, 1, config=96)[0]
    x, info = P.solve(torch.from_numpy(b).to(DEV), tol=1e-12, preconditioner=amg.PC_AMGR)
    assert info.converged
    assert _rel(x.cpu().numpy(), spla.spsolve(A.tocsc(), b)) <= 1e-8
    Q = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64)
    with pytest.raises(amg.AmgsymError) as e:
        Q.solve(torch.from_numpy(b).to(DEV), preconditioner=amg.PC_AMGR)
    assert e.value.name == "ERR_STATE"


def test_model_problem_amgr_beats_the_inner_block_amg():
    N = (32, 32, 32)
    h = grid.widths(N, 1.5)
    rows = {}
    for s in range(4):
        P = amg.Problem.structured(N, 1.5, None, s, bc="neumann").setup(amgr=1)
        f = np.random.default_rng(97).uniform(-1.0, 1.0, P.n)
        b = f * fv.cell_volumes(h)
        b -= b.mean()
        bt = torch.from_numpy(b).to(DEV)
        x, ia = P.solve(bt, tol=1e-8, preconditioner=amg.PC_AMGR)
        assert ia.converged
        r = b - fv.apply(h, np.ones(P.n), x.cpu().numpy(), "neumann")
        assert np.linalg.norm(r) <= 1.05e-8 * np.linalg.norm(b)
        _, im = P.solve(bt, tol=1e-8)
        rows[s] = (ia.iters, im.iters)
        if s >= 1:
            assert ia.iters < im.iters, (s, rows[s])
    print("PCG iterations (AMGR, I (x) M_inn^-1) by s:", rows)


def test_profile_step_with_amgr_times_its_launches():
    """amgsym_profile_step with the AMGR preconditioner: the step's records
    include AMGR's own launches (top smoother, restriction to the coarse
    domain, the AMG of A_c) and leave the solve's result unchanged."""
    N, s = (32, 32, 32), 3
    P = amg.Problem.structured(N, 1.5, None, s).setup(amgr=1)
    b = torch.from_numpy(rhs_uniform(P.n, 1, config=97)).to(DEV)
    x1, i1 = P.solve(b, tol=1e-10, precision=amg.PREC_MIXED_FP32, preconditioner=amg.PC_AMGR)
    recs = P.profile_step(b, torch.empty_like(b), 1, amg.PREC_MIXED_FP32, preconditioner=amg.PC_AMGR)
    roles = [r["role"] for r in recs if r["phase"] == 1]
    assert any("AMGR coarse-point smoother" in r for r in roles)
    assert all(r["us"] > 0 for r in recs)
    x2, i2 = P.solve(b, tol=1e-10, precision=amg.PREC_MIXED_FP32, preconditioner=amg.PC_AMGR)
    assert i1.iters == i2.iters and torch.equal(x1, x2)
    Q = amg.Problem.structured(N, 1.5, None, s).setup()
    with pytest.raises(amg.AmgsymError):
        Q.profile_step(b, torch.empty_like(b), 1, amg.PREC_MIXED_FP32, preconditioner=amg.PC_AMGR)


@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_transformed_basis_coarse_operator_equals_the_assembled_one(prec):
    """opts.amgr_sym_ac: the coarse problem's level-0 products with A_c run as
    butterfly -> reduced SpMM (P_b^T A_inn P_b read once, coarse couplings)
    -> scaled butterfly (eq. "structAc" under eq. "P_s").  The same operator
    to rounding: AMGR applications agree with those of the assembled A_c, and
    the solves converge alike."""
    N, s = (24, 20, 16), 3
    g = gaussian_logk(N, s, seed=98, corr=2.0)
    P1 = amg.Problem.structured(N, 1.5, g, s).setup(amgr=1, amgr_sym_ac=1, coarse_max=64)
    P0 = amg.Problem.structured(N, 1.5, g, s).setup(amgr=1, amgr_sym_ac=0, coarse_max=64)
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    U = torch.from_numpy(np.random.default_rng(9).standard_normal((P1.n_b, 2 << s))).to(DEV, dt)
    Z1, Z0 = torch.empty_like(U), torch.empty_like(U)
    P1.amgr_apply(U, Z1, 2, prec)
    P0.amgr_apply(U, Z0, 2, prec)
    d = (Z1 - Z0).double().norm() / Z0.double().norm()
    assert d <= (1e-12 if prec == amg.PREC_FP64 else 1e-5), float(d)
    b = torch.from_numpy(rhs_uniform(P1.n, 1, config=99)).to(DEV)
    x1, i1 = P1.solve(b, tol=1e-10, precision=prec, preconditioner=amg.PC_AMGR)
    x0, i0 = P0.solve(b, tol=1e-10, precision=prec, preconditioner=amg.PC_AMGR)
    assert i1.converged and i0.converged and abs(i1.iters - i0.iters) <= 1
    assert (x1 - x0).norm() <= 1e-8 * x0.norm()
    roles = [r["role"] for r in P1.profile_step(b, torch.empty_like(b), 1, amg.PREC_MIXED_FP32,
                                                 preconditioner=amg.PC_AMGR)]
    assert any("AMGR A_c: to the transformed basis" in r for r in roles)
    roles0 = [r["role"] for r in P0.profile_step(b, torch.empty_like(b), 1, amg.PREC_MIXED_FP32,
                                                  preconditioner=amg.PC_AMGR)]
    assert not any("AMGR A_c" in r for r in roles0)
