"""The diagonal-offset storage of the finest-level stencil and its FSAI
factors (marked gpu): products in that form equal the CSR products bit for
bit (same values, same summation order), so the reduced operator and the
V-cycle are identical with and without it, and solves agree to rounding of
their dot products (whose block partition follows each kernel's grid)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from gpu_common import oracle_apply_hat, oracle_hat_blocks, oracle_problem  # noqa: E402
from synth import batched_problem_specs, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [
    ((30, 22, 18), 3, 1),  # C = 8: two 16-byte vectors per thread
    ((20, 14, 10), 2, 3),  # C = 12: one vector per thread
    ((40, 36), 1, 2),      # 2-D, 5 diagonals
    ((12, 10, 8), 0, 3),   # no symmetry, C = 3: scalar columns
]


def _pair(N, s, precisions=3):
    g, h, k, A = oracle_problem(N, s, 1.5, True)
    P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, precisions=precisions)
    Q = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, precisions=precisions, dia_max_diag=0)
    assert P.level_dia(0, "A")["ndiag"] == 2 * len(N) + 1
    assert Q.level_dia(0, "A")["ndiag"] == 0
    return P, Q, A


@pytest.mark.parametrize("N,s,nrhs", CASES)
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_reduced_operator_bit_identical_and_matches_oracle(N, s, nrhs, prec):
    P, Q, A = _pair(N, s)
    C = nrhs << s
    X = np.random.default_rng(11).uniform(-1, 1, (P.n_b, C))
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    Xt = torch.from_numpy(X).to(DEV, dt)
    Y1, Y2 = torch.empty_like(Xt), torch.empty_like(Xt)
    P.apply_reduced(Xt, Y1, nrhs, prec)
    Q.apply_reduced(Xt, Y2, nrhs, prec)
    assert torch.equal(Y1, Y2)
    perm, hat = oracle_hat_blocks(A, N, s)
    Yref = oracle_apply_hat(hat, Xt.double().cpu().numpy(), 1 << s)
    tol = 1e-14 if prec == amg.PREC_FP64 else 1e-6
    assert np.max(np.abs(Y1.double().cpu().numpy() - Yref)) <= tol * np.max(np.abs(A.data)) * 8


@pytest.mark.parametrize("N,s,nrhs", CASES)
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32, amg.PREC_MIXED_BF16])
def test_vcycle_bit_identical(N, s, nrhs, prec):
    P, Q, A = _pair(N, s, precisions=7)
    C = nrhs << s
    R = np.random.default_rng(12).uniform(-1, 1, (P.n_b, C))
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    Rt = torch.from_numpy(R).to(DEV, dt)
    Z1, Z2 = torch.empty_like(Rt), torch.empty_like(Rt)
    P.vcycle(Rt, Z1, nrhs, prec)
    Q.vcycle(Rt, Z2, nrhs, prec)
    assert torch.equal(Z1, Z2)
    assert torch.isfinite(Z1).all()


@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_solve_agrees(prec):
    N, s = (30, 22, 18), 3
    P, Q, A = _pair(N, s)
    b = torch.from_numpy(rhs_uniform(P.n, 2, config=21)).to(DEV)
    x1, r1 = P.solve(b, tol=1e-10, precision=prec)
    x2, r2 = Q.solve(b, tol=1e-10, precision=prec)
    assert r1.converged and r2.converged
    assert abs(r1.iters - r2.iters) <= 1
    d = (x1 - x2).norm() / x2.norm()
    assert d.item() <= 1e-8


def test_batched_agrees():
    specs = batched_problem_specs(count=4, nmin=16, nmax=32)
    on, off, bs = [], [], []
    for k, sp in enumerate(specs):
        on.append(amg.Problem.structured(sp["N"], 0.0, None, sp["s"]).setup(coarse_max=64))
        off.append(amg.Problem.structured(sp["N"], 0.0, None, sp["s"]).setup(coarse_max=64, dia_max_diag=0))
        bs.append(torch.from_numpy(rhs_uniform(on[-1].n, 4, config=600 + k)).to(DEV))
    x1, r1 = amg.Batch(on, [4] * 4).solve(bs, tol=1e-10)
    x2, r2 = amg.Batch(off, [4] * 4).solve(bs, tol=1e-10)
    for p in range(4):
        assert r1[p].converged and r2[p].converged
        assert ((x1[p] - x2[p]).norm() / x2[p].norm()).item() <= 1e-8
