"""The persistent coarse-cycle kernel (marked gpu): the V-cycle levels from
fuse_rows down run as the phases of one cooperative launch with grid
barriers.  Its phases are the stand-alone products with the same arguments
and entry lanes, so V-cycles and whole solves equal the one-launch-per-product
path bit for bit; its bounded barrier wait ends with a reported error and a
usable handle when nothing releases it."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from gpu_common import oracle_problem  # noqa: E402
from synth import rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [
    ((32, 28, 24), 3, 1),  # C = 8
    ((24, 20, 16), 2, 3),  # C = 12
    ((48, 40), 1, 2),      # 2-D, C = 4
    ((14, 12, 10), 0, 3),  # C = 3: scalar columns
]


def _pair(N, s, fuse_rows=1 << 30, **kw):
    g, h, k, A = oracle_problem(N, s, 1.5, True)
    P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=32, precisions=7, fuse_rows=fuse_rows, **kw)
    Q = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=32, precisions=7, fuse_rows=0, **kw)
    assert P.num_levels() >= 3
    return P, Q


@pytest.mark.parametrize("N,s,nrhs", CASES)
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32, amg.PREC_MIXED_BF16])
def test_vcycle_bit_identical(N, s, nrhs, prec):
    P, Q = _pair(N, s)
    C = nrhs << s
    R = np.random.default_rng(3).uniform(-1, 1, (P.n_b, C))
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    Rt = torch.from_numpy(R).to(DEV, dt)
    Z1, Z2 = torch.empty_like(Rt), torch.empty_like(Rt)
    for _ in range(2):  # the second call replays the cached plan
        P.vcycle(Rt, Z1, nrhs, prec)
        Q.vcycle(Rt, Z2, nrhs, prec)
        assert torch.equal(Z1, Z2)
    assert torch.isfinite(Z1).all()


@pytest.mark.parametrize("fuse_rows", [1 << 30, 300])
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_solve_bit_identical(fuse_rows, prec):
    """Whole solves (graph replay, look-ahead, refinement) give the same
    iterates: fused from level 1 down, or from a deeper level."""
    N, s = (32, 28, 24), 3
    P, Q = _pair(N, s, fuse_rows=fuse_rows)
    b = torch.from_numpy(rhs_uniform(P.n, 2, config=31)).to(DEV)
    x1, r1 = P.solve(b, tol=1e-10, precision=prec)
    x2, r2 = Q.solve(b, tol=1e-10, precision=prec)
    x3, r3 = P.solve(b, tol=1e-10, precision=prec, use_graph=0)
    assert r1.converged and r1.iters == r2.iters == r3.iters
    assert torch.equal(x1, x2) and torch.equal(x1, x3)


def test_barrier_timeout_is_reported_and_handle_stays_usable():
    N, s = (32, 28, 24), 3
    P, Q = _pair(N, s)
    b = torch.from_numpy(rhs_uniform(P.n, 1, config=32)).to(DEV)
    x0, _ = P.solve(b, tol=1e-10, precision=amg.PREC_MIXED_FP32)
    P.cycle_timeout_check(1, amg.PREC_MIXED_FP32)   # raises unless the timeout was reported
    x1, r1 = P.solve(b, tol=1e-10, precision=amg.PREC_MIXED_FP32)
    assert r1.converged and torch.equal(x0, x1)
    with pytest.raises(amg.AmgsymError):
        Q.cycle_timeout_check(1, amg.PREC_MIXED_FP32)  # no fused cycle on this handle
