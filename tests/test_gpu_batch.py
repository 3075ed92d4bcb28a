"""Batched solve (marked gpu): many problems of uneven sizes, symmetry
counts and RHS counts in one pass, each checked against the oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from oracle import fv, grid, solvers  # noqa: E402
from synth import batched_problem_specs, gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

MIXED = [((24, 24, 24), 3, 16, 0.0, False), ((40, 24, 16), 1, 3, 0.0, False), ((32, 32, 32), 2, 16, 1.5, True),
         ((20, 18, 16), 1, 1, 1.5, True), ((48, 32, 32), 3, 2, 0.0, False), ((16, 16, 16), 2, 5, 0.0, False)]


def _build(cases, coarse_max=64):
    probs, bs, refs = [], [], []
    for k, (N, s, nrhs, gamma, vark) in enumerate(cases):
        g = gaussian_logk(N, s, seed=40 + k, corr=3.0) if vark else None
        P = amg.Problem.structured(N, gamma, g, s).setup(coarse_max=coarse_max, precisions=7)
        b = rhs_uniform(P.n, nrhs, config=20 + k)
        probs.append(P)
        bs.append(b)
        if vark:
            h, kk, A = fv.grid_operator(N, gamma, g)
            import scipy.sparse.linalg as spla

            lu = spla.splu(A.tocsc())
            refs.append(np.stack([lu.solve(bi) for bi in b]))
        else:
            refs.append(solvers.dst_solve(N, b).reshape(nrhs, -1))
    return probs, bs, refs


@pytest.mark.parametrize("prec", [amg.PREC_MIXED_FP32, amg.PREC_MIXED_BF16])
def test_batch_matches_oracle(prec):
    probs, bs, refs = _build(MIXED)
    B = amg.Batch(probs, [b.shape[0] for b in bs])
    xs, res = B.solve([torch.from_numpy(b).to(DEV) for b in bs], tol=1e-10, precision=prec)
    torch.cuda.synchronize()
    for p in range(len(probs)):
        assert res[p].converged, (p, res[p])
        assert np.all(res[p].relres <= 1e-10)
        x = xs[p].cpu().numpy()
        for r in range(x.shape[0]):
            err = np.linalg.norm(x[r] - refs[p][r]) / np.linalg.norm(refs[p][r])
            assert err <= 1e-6, (p, r, err)


def test_batch_equals_single_problem_solves_and_repeats():
    probs, bs, refs = _build(MIXED[:4])
    B = amg.Batch(probs, [b.shape[0] for b in bs])
    bt = [torch.from_numpy(b).to(DEV) for b in bs]
    xs1, res1 = B.solve(bt, tol=1e-10)
    xs2, res2 = B.solve(bt, tol=1e-10)  # graph replay on the second call
    for p in range(len(probs)):
        assert torch.equal(xs1[p], xs2[p])
        xsingle, info = probs[p].solve(bt[p], tol=1e-10, precision=amg.PREC_MIXED_FP32)
        a = xs1[p].cpu().numpy()
        c = xsingle.cpu().numpy()
        assert np.linalg.norm(a - c) <= 1e-7 * np.linalg.norm(c)


def test_batch_recipe_sample_residuals():
    """The batched workload's recipe (even N, s in {1,2,3}, 16 RHS), with the
    cube edge drawn from [32, 64] to keep the oracle check short: every
    problem's true residual checked with the oracle's own operator."""
    specs = batched_problem_specs(count=6, nmin=32, nmax=64)
    probs, bs = [], []
    for k, sp in enumerate(specs):
        P = amg.Problem.structured(sp["N"], 0.0, None, sp["s"]).setup()
        probs.append(P)
        bs.append(rhs_uniform(P.n, 16, config=400 + k))
    B = amg.Batch(probs, [16] * len(probs))
    xs, res = B.solve([torch.from_numpy(b).to(DEV) for b in bs], tol=1e-8)
    for p, sp in enumerate(specs):
        assert res[p].converged
        h = grid.widths(sp["N"], 0.0)
        x = xs[p].cpu().numpy()
        for r in range(16):
            rr = bs[p][r] - fv.apply(h, np.ones(probs[p].n), x[r])
            assert np.linalg.norm(rr) / np.linalg.norm(bs[p][r]) <= 1.05e-8
