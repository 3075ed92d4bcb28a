"""New coefficient values on a set-up problem (marked gpu).

amgsym_update_values frees the device copies of the hierarchy; the device
path must then refuse to solve until amgsym_setup has run again, and after it
solve the new operator, alone and inside a batch that was created before the
update (its launch plans and captured graph pointed at the freed copies)."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from oracle import fv, grid, symmetry  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _operator(N, s, seed):
    g = gaussian_logk(N, s, seed=seed, corr=2.0)
    return fv.assemble(grid.widths(N, 1.5), np.exp(g))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_update_values_then_setup_solves_the_new_operator():
    N, s = (24, 20, 16), 3
    A1, A2 = _operator(N, s, 31), _operator(N, s, 32)
    P = amg.Problem(A1.shape[0], A1.indptr, A1.indices, A1.data, s, symmetry.mirror_perm(N, s))
    P.setup(coarse_max=64)
    b = rhs_uniform(P.n, 2, config=60)
    bt = torch.from_numpy(b).to(DEV)
    x1, info = P.solve(bt, tol=1e-12)
    assert info.converged
    lu1 = spla.splu(A1.tocsc())
    for r in range(2):
        assert _rel(x1[r].cpu().numpy(), lu1.solve(b[r])) <= 1e-8
    P.update_values(A2.data)
    with pytest.raises(amg.AmgsymError) as e:
        P.solve(bt, tol=1e-12)
    assert e.value.name == "ERR_STATE"
    P.setup(coarse_max=64)
    lu2 = spla.splu(A2.tocsc())
    for prec, tol, bound in ((amg.PREC_FP64, 1e-12, 1e-8), (amg.PREC_MIXED_FP32, 1e-10, 1e-6)):
        x2, info = P.solve(bt, tol=tol, precision=prec)
        assert info.converged and np.all(info.relres <= tol)
        for r in range(2):
            assert _rel(x2[r].cpu().numpy(), lu2.solve(b[r])) <= bound


def test_batch_created_before_an_update_rebuilds_its_plans():
    cases = [((24, 24, 16), 3, 31, 4), ((20, 16, 16), 1, 33, 2)]
    probs, bs, ops = [], [], []
    for k, (N, s, seed, nrhs) in enumerate(cases):
        A = _operator(N, s, seed)
        P = amg.Problem(A.shape[0], A.indptr, A.indices, A.data, s, symmetry.mirror_perm(N, s))
        P.setup(coarse_max=64)
        probs.append(P)
        ops.append(A)
        bs.append(rhs_uniform(P.n, nrhs, config=70 + k))
    B = amg.Batch(probs, [b.shape[0] for b in bs])
    bt = [torch.from_numpy(b).to(DEV) for b in bs]
    B.solve(bt, tol=1e-10)  # builds the plans and captures the graph
    # new coefficients for problem 0, a new hierarchy; problem 1 unchanged
    N0, s0 = cases[0][0], cases[0][1]
    A0 = _operator(N0, s0, 35)
    probs[0].update_values(A0.data)
    probs[0].setup(coarse_max=64)
    ops[0] = A0
    for _ in range(2):  # the rebuild, then a replay of the rebuilt graph
        xs, res = B.solve(bt, tol=1e-10)
        torch.cuda.synchronize()
        for p in range(len(probs)):
            assert res[p].converged, (p, res[p])
            lu = spla.splu(ops[p].tocsc())
            x = xs[p].cpu().numpy()
            for r in range(x.shape[0]):
                assert _rel(x[r], lu.solve(bs[p][r])) <= 1e-6, (p, r)
    # a problem set up into a single level no longer fits a batch
    probs[1].update_values(ops[1].data)
    probs[1].setup(coarse_max=4096)
    with pytest.raises(amg.AmgsymError) as e:
        B.solve(bt, tol=1e-10)
    assert e.value.name == "ERR_STATE"
