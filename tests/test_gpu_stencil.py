"""The z-marching stencil kernel of the finest-level diagonal-offset products
(opts.zmarch; marked gpu).

The stencil kernel addresses every neighbour by its row index, like the
diagonal-offset kernel, so its products must be bit-identical to it: the
reduced operator A^ (eq. "hL_splitting", interface couplings included) and
the V-cycle, which runs the finest-level A, G and G^T products through it.
The cases cut the (tile, plane) units so that blocks' ranges cross tiles
(restarts of the march) and include BF16 matrix values.  The solve through
it meets the oracle, and the profile names the kernel it ran.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from oracle import fv, solvers  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

# (N, s, nrhs): 8 columns; base blocks 32^3 (one tile across, 32 planes) and
# 64^3 and 64 x 64 x 32 (16 and 8 tiles: ranges of a few planes cross tiles)
CASES = [((64, 64, 64), 3, 1), ((128, 128, 128), 3, 1), ((128, 128, 64), 3, 1), ((64, 64, 64), 2, 2)]


def _pair(N, s, vark, gamma=1.5, **kw):
    g = gaussian_logk(N, s, seed=71, corr=4.0) if vark else None
    P1 = amg.Problem.structured(N, gamma, g, s).setup(zmarch=1, **kw)
    P0 = amg.Problem.structured(N, gamma, g, s).setup(zmarch=0, **kw)
    return P1, P0


@pytest.mark.parametrize("N,s,nrhs", CASES)
@pytest.mark.parametrize("prec", [amg.PREC_MIXED_FP32, amg.PREC_MIXED_BF16])
def test_reduced_operator_and_vcycle_bit_identical(N, s, nrhs, prec):
    kw = dict(precisions=7) if prec == amg.PREC_MIXED_BF16 else {}
    P1, P0 = _pair(N, s, True, **kw)
    C = nrhs * P1.nb
    X = torch.randn((P1.n_b, C), dtype=torch.float32, device=DEV)
    Y1 = torch.empty_like(X)
    Y0 = torch.empty_like(X)
    P1.apply_reduced(X, Y1, nrhs, prec)
    P0.apply_reduced(X, Y0, nrhs, prec)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y0)
    Z1 = torch.empty_like(X)
    Z0 = torch.empty_like(X)
    P1.vcycle(X, Z1, nrhs, prec)
    P0.vcycle(X, Z0, nrhs, prec)
    torch.cuda.synchronize()
    assert torch.equal(Z1, Z0)
    assert torch.isfinite(Z1).all() and Z1.abs().max() > 0


def test_solve_runs_the_stencil_kernel_and_meets_the_oracle():
    N, s = (64, 64, 64), 3
    P1, P0 = _pair(N, s, False, gamma=0.0)  # uniform grid: the DST closed form is the oracle
    b = rhs_uniform(P1.n, 1, config=72)
    x1, i1 = P1.solve(torch.from_numpy(b).to(DEV), tol=1e-10, precision=amg.PREC_MIXED_FP32)
    x0, i0 = P0.solve(torch.from_numpy(b).to(DEV), tol=1e-10, precision=amg.PREC_MIXED_FP32)
    xo = solvers.dst_solve(N, b)
    for x in (x1, x0):
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    # the fused dots sum the rows in another grouping: iteration counts agree closely
    assert abs(i1.iters - i0.iters) <= 2
    bt = torch.from_numpy(b).to(DEV)
    names1 = {r["kernel"].split("<")[0] for r in P1.profile_step(bt, torch.empty_like(bt), 1, amg.PREC_MIXED_FP32)}
    names0 = {r["kernel"].split("<")[0] for r in P0.profile_step(bt, torch.empty_like(bt), 1, amg.PREC_MIXED_FP32)}
    assert "stencil_kernel" in names1 and "stencil_kernel" not in names0


def test_grid_that_does_not_fit_the_tiles_uses_the_diagonal_kernel():
    # base block 24 x 24 x 24: the first stride is not a multiple of 32
    N, s = (48, 48, 48), 3
    P = amg.Problem.structured(N, 1.5, None, s).setup(zmarch=1)
    b = rhs_uniform(P.n, 1, config=73)
    bt = torch.from_numpy(b).to(DEV)
    names = {r["kernel"].split("<")[0] for r in P.profile_step(bt, torch.empty_like(bt), 1, amg.PREC_MIXED_FP32)}
    assert "stencil_kernel" not in names
    x, info = P.solve(bt, tol=1e-10, precision=amg.PREC_MIXED_FP32)
    r = b - fv.apply(P.grid["widths"], P.grid["k"], x.cpu().numpy()[0], "dirichlet")
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)
