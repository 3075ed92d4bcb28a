"""The sliced (SELL-32) form of the hierarchy's CSR matrices (opts.sell;
marked gpu).

A sliced product keeps, per row, the CSR kernel's entry-lane partial sums
and their combination order, so a V-cycle and a whole solve with it must
give the same bits as with the CSR kernel alone, in every precision whose
tile runs one vector of C columns per thread (FP32 and BF16 values at 8
columns, FP64 at 4).  The profile names the kernel that ran.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from oracle import solvers  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _pair(N, s, gamma=1.5, vark=True, **kw):
    g = gaussian_logk(N, s, seed=81, corr=3.0) if vark else None
    P = amg.Problem.structured(N, gamma, g, s).setup(sell=1, precisions=7, **kw)
    Q = amg.Problem.structured(N, gamma, g, s).setup(sell=0, precisions=7, **kw)
    return P, Q


# (N, s, nrhs, prec): 8 FP32 columns (s = 3; s = 2 with 2 RHS), 4 FP64 columns
CASES = [
    ((64, 64, 64), 3, 1, amg.PREC_MIXED_FP32),
    ((64, 64, 64), 3, 1, amg.PREC_MIXED_BF16),
    ((64, 48, 40), 2, 2, amg.PREC_MIXED_FP32),
    ((64, 48, 40), 2, 1, amg.PREC_FP64),
]


@pytest.mark.parametrize("N,s,nrhs,prec", CASES)
def test_vcycle_bit_identical(N, s, nrhs, prec):
    P, Q = _pair(N, s)
    C = nrhs << s
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    R = torch.from_numpy(np.random.default_rng(8).uniform(-1, 1, (P.n_b, C))).to(DEV, dt)
    Z1, Z2 = torch.empty_like(R), torch.empty_like(R)
    for _ in range(2):
        P.vcycle(R, Z1, nrhs, prec)
        Q.vcycle(R, Z2, nrhs, prec)
        torch.cuda.synchronize()
        assert torch.equal(Z1, Z2)
    assert torch.isfinite(Z1).all()


@pytest.mark.parametrize("prec", [amg.PREC_MIXED_FP32, amg.PREC_FP64])
def test_solve_bit_identical_and_sliced_kernel_used(prec):
    N, s = ((64, 64, 64), 3) if prec != amg.PREC_FP64 else ((64, 48, 40), 2)
    P, Q = _pair(N, s)
    b = torch.from_numpy(rhs_uniform(P.n, 1, config=82)).to(DEV)
    # fixed tiles: the autotuner times what runs, so it may pick another
    # entry-lane count (another summation grouping) with the sliced form
    x1, i1 = P.solve(b, tol=1e-10, precision=prec, tune=0)
    x2, i2 = Q.solve(b, tol=1e-10, precision=prec, tune=0)
    assert i1.converged and i1.iters == i2.iters and torch.equal(x1, x2)
    k1 = [r for r in P.profile_step(b, torch.empty_like(b), 1, prec) if r["kernel"].startswith("sell_kernel")]
    k2 = [r for r in Q.profile_step(b, torch.empty_like(b), 1, prec) if r["kernel"].startswith("sell_kernel")]
    assert k1 and not k2
    assert any(r["role"].startswith("L1 A") for r in k1)


def test_sliced_solve_meets_the_oracle():
    N, s = (64, 64, 64), 3
    P, _ = _pair(N, s, gamma=0.0, vark=False)
    b = rhs_uniform(P.n, 1, config=83)
    x, info = P.solve(torch.from_numpy(b).to(DEV), tol=1e-10, precision=amg.PREC_MIXED_FP32)
    xo = solvers.dst_solve(N, b)
    assert info.converged
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)
