"""Differentiable solve (marked gpu): the autograd adjoint against the
oracle's dense adjoint and against central finite differences of the
oracle's unreduced solve (a symmetry-breaking perturbation cannot use the
reduced solve, so the FD reference must be the full system)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from paper_2407_05930_gb300.autograd import sym_poisson_solve  # noqa: E402
from oracle import adjoint, fv, grid  # noqa: E402
from synth import CONFIGS, gaussian_logk, rhs_uniform, u_target  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _grads(N, s, gamma, prec=amg.PREC_FP64, tol=1e-12, seed=5):
    g = gaussian_logk(N, s, seed=seed, corr=3.0)
    n = int(np.prod(N))
    b = rhs_uniform(n, 1, config=5)[0]
    ut = u_target(n)
    bt = torch.from_numpy(b).to(DEV).requires_grad_(True)
    gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
    u = sym_poisson_solve(bt, gt, N, gamma, s, solve_kw=dict(tol=tol, precision=prec))
    L = torch.sum((u - torch.from_numpy(ut).to(DEV)) ** 2)
    L.backward()
    return g, b, ut, float(L), bt.grad.cpu().numpy(), gt.grad.cpu().numpy()


def test_adjoint_matches_oracle_and_fd_32cube():
    N, s, gamma = (32, 32, 32), 3, 1.5
    g, b, ut, L, db, dg = _grads(N, s, gamma)
    h = grid.widths(N, gamma)
    Lo, dbo, dgo = adjoint.gradients(h, g, b, ut)
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    assert np.linalg.norm(db - dbo) <= 1e-8 * np.linalg.norm(dbo)
    assert np.linalg.norm(dg - dgo) <= 1e-8 * np.linalg.norm(dgo)
    # central differences of the oracle's unreduced loss, random directions
    rng = np.random.default_rng(17)
    eps = 1e-6
    v = rng.standard_normal(g.size)
    fd = (adjoint.loss(h, g + eps * v, b, ut) - adjoint.loss(h, g - eps * v, b, ut)) / (2 * eps)
    assert abs(fd - dg @ v) <= 1e-6 * abs(fd)
    w = rng.standard_normal(b.size)
    fd = (adjoint.loss(h, g, b + eps * w, ut) - adjoint.loss(h, g, b - eps * w, ut)) / (2 * eps)
    assert abs(fd - db @ w) <= 1e-6 * abs(fd)


def test_adjoint_mixed_precision_small():
    N, s, gamma = (24, 16, 16), 2, 1.5
    g, b, ut, L, db, dg = _grads(N, s, gamma, prec=amg.PREC_MIXED_FP32, tol=1e-10)
    h = grid.widths(N, gamma)
    Lo, dbo, dgo = adjoint.gradients(h, g, b, ut)
    assert np.linalg.norm(dg - dgo) <= 1e-6 * np.linalg.norm(dgo)
    assert np.linalg.norm(db - dbo) <= 1e-6 * np.linalg.norm(dbo)


def test_adjoint_full_size_192cube_mixed():
    """192^3 stretched variable-coefficient problem, mixed precision at the
    workload tolerance: the oracle's own operator confirms the forward and
    adjoint residuals; the gradient kernel is pinned at small sizes."""
    cfg = CONFIGS[5]
    N, s = cfg["N"], cfg["s"]
    g = gaussian_logk(N, s, seed=5000, corr=8.0)
    n = int(np.prod(N))
    b = rhs_uniform(n, 1, config=5)[0]
    ut = u_target(n)
    bt = torch.from_numpy(b).to(DEV).requires_grad_(True)
    gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
    u = sym_poisson_solve(bt, gt, N, 1.5, s, solve_kw=dict(tol=cfg["tol"], precision=amg.PREC_MIXED_FP32))
    utt = torch.from_numpy(ut).to(DEV)
    L = torch.sum((u - utt) ** 2)
    L.backward()
    h = grid.widths(N, 1.5)
    k = np.exp(g)
    uu = u.detach().cpu().numpy()
    assert np.linalg.norm(b - fv.apply(h, k, uu)) / np.linalg.norm(b) <= 1.05 * cfg["tol"]
    lam = bt.grad.cpu().numpy()
    rhs = 2.0 * (uu - ut)
    assert np.linalg.norm(rhs - fv.apply(h, k, lam)) / np.linalg.norm(rhs) <= 1.05 * cfg["tol"]
    dg = gt.grad.cpu().numpy()
    assert np.all(np.isfinite(dg))
    # gradient formula applied by the oracle to the GPU's u and lambda
    ref = adjoint.grad_logk(h, k, uu, lam)
    assert np.linalg.norm(dg - ref) <= 1e-10 * np.linalg.norm(ref)


def test_second_forward_reuses_the_handle():
    """An optimisation loop: two forwards with different fields on one
    SymPoisson create one problem (the second field goes through
    amgsym_update_values), and both gradients match the oracle's."""
    from paper_2407_05930_gb300.autograd import SymPoisson

    N, s, gamma = (32, 32, 32), 3, 1.5
    op = SymPoisson(N, gamma, s, solve_kw=dict(tol=1e-12, precision=amg.PREC_FP64))
    n = int(np.prod(N))
    b = rhs_uniform(n, 1, config=5)[0]
    ut = u_target(n)
    h = grid.widths(N, gamma)
    handle = None
    for seed in (5, 6):
        g = gaussian_logk(N, s, seed=seed, corr=3.0)
        bt = torch.from_numpy(b).to(DEV).requires_grad_(True)
        gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
        u = op(bt, gt)
        L = torch.sum((u - torch.from_numpy(ut).to(DEV)) ** 2)
        L.backward()
        if handle is None:
            handle = op.P._h.value
        assert op.P._h.value == handle and op.creates == 1
        Lo, dbo, dgo = adjoint.gradients(h, g, b, ut)
        assert abs(float(L) - Lo) <= 1e-9 * abs(Lo)
        assert np.linalg.norm(bt.grad.cpu().numpy() - dbo) <= 1e-8 * np.linalg.norm(dbo)
        assert np.linalg.norm(gt.grad.cpu().numpy() - dgo) <= 1e-8 * np.linalg.norm(dgo)
    assert op.setups == 2
    # a forward with the first field again, then both backwards in reverse
    # order: each backward solves with its own forward's operator
    g5, g6 = gaussian_logk(N, s, seed=5, corr=3.0), gaussian_logk(N, s, seed=6, corr=3.0)
    outs = []
    for g in (g5, g6):
        gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
        u = op(torch.from_numpy(b).to(DEV), gt)
        outs.append((g, gt, torch.sum((u - torch.from_numpy(ut).to(DEV)) ** 2)))
    for g, gt, L in reversed(outs):
        L.backward()
        _, _, dgo = adjoint.gradients(h, g, b, ut)
        assert np.linalg.norm(gt.grad.cpu().numpy() - dgo) <= 1e-8 * np.linalg.norm(dgo)
    assert op.creates == 1
