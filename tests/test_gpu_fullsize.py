"""Parity at the benchmark's full sizes (marked gpu).

At 256^3 with three symmetries the oracle transforms the whole vector (its
butterfly is vectorised) and evaluates sampled rows of the reduced operator
one by one from the assembled matrix; the batched workload at its full recipe
(64 problems, N in [32, 160], 16 RHS) is checked through true residuals with
the oracle's own operator on sampled problems."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from gpu_common import oracle_forward  # noqa: E402
from oracle import fv, grid, symmetry, transform  # noqa: E402
from synth import CONFIGS, batched_problem_specs, gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def big():
    """The 256^3 stretched-grid variable-k problem (k = exp of the smoothed
    mirror-symmetric field, seed 3000, correlation 8 cells)."""
    cfg = CONFIGS[3]
    N, s, gamma = cfg["N"], cfg["s"], cfg["gamma"]
    g = gaussian_logk(N, s, seed=3000, corr=8.0)
    P = amg.Problem.structured(N, gamma, g, s).setup(precisions=3)
    h, k, A = fv.grid_operator(N, gamma, g)
    return P, A, symmetry.mirror_perm(N, s), N, s


def test_transform_full_256cube(big):
    P, A, perm, N, s = big
    b = rhs_uniform(P.n, 1, config=3)
    xh = torch.empty((P.n_b, 1 << s), dtype=torch.float64, device=DEV)
    P.transform_forward(torch.from_numpy(b).to(DEV), 1, xh)
    ref = oracle_forward(b, N, s)
    assert np.max(np.abs(xh.cpu().numpy() - ref)) <= 1e-14 * np.max(np.abs(ref))
    back = torch.empty((1, P.n), dtype=torch.float64, device=DEV)
    P.transform_backward(xh, 1, back)
    assert np.max(np.abs(back.cpu().numpy() - b)) <= 1e-15


def _sample_rows(n_b, perm, N, seed):
    """Random rows plus rows next to each mirror plane (the ones with an
    interface coupling A_out) and the first and last row."""
    rng = np.random.default_rng(seed)
    rows = rng.choice(n_b, size=1500, replace=False)
    base = np.array(N) // 2
    nx, ny = base[0], base[1]
    l = np.arange(n_b)
    ix, iy, iz = l % nx, (l // nx) % ny, l // (nx * ny)
    plane = np.flatnonzero((ix == nx - 1) | (iy == ny - 1) | (iz == base[2] - 1))
    return np.unique(np.concatenate([rows, rng.choice(plane, size=500, replace=False), [0, n_b - 1]]))


@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_reduced_operator_sampled_rows_256cube(big, prec):
    """Sampled rows of Y[:, i] = A^_i X[:, i] with A^_i = sum_j sign(i, j) H_j
    (the decoupled blocks of the transformed operator), each row built from
    the row of A for the base cell: column q of that row lies in copy j(q) at
    base index k(q), and contributes sign(i, j(q)) a_q X[k(q), i]."""
    P, A, perm, N, s = big
    nb = 1 << s
    X = np.random.default_rng(1).uniform(-1, 1, (P.n_b, nb))
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    Xt = torch.from_numpy(X).to(DEV, dt)
    Yt = torch.empty_like(Xt)
    P.apply_reduced(Xt, Yt, 1, prec)
    Y = Yt.double().cpu().numpy()
    Xr = Xt.double().cpu().numpy()  # the operand the kernel saw
    flat = perm.reshape(-1)
    base_of = np.empty(P.n, dtype=np.int64)
    base_of[flat] = np.arange(P.n) % P.n_b
    copy_of = np.empty(P.n, dtype=np.int64)
    copy_of[flat] = np.arange(P.n) // P.n_b
    sign = np.array([[transform.hadamard_sign(i, j) for j in range(nb)] for i in range(nb)])
    rows = _sample_rows(P.n_b, perm, N, seed=2)
    scale = np.max(np.abs(A.data))
    tol = 1e-14 if prec == amg.PREC_FP64 else 1e-6
    worst = 0.0
    for l in rows:
        p = perm[0, l]
        cols = A.indices[A.indptr[p]:A.indptr[p + 1]]
        vals = A.data[A.indptr[p]:A.indptr[p + 1]]
        ref = np.zeros(nb)
        for q, a in zip(cols, vals):
            ref += sign[:, copy_of[q]] * a * Xr[base_of[q]]
        worst = max(worst, float(np.max(np.abs(Y[l] - ref))))
    assert worst <= tol * scale * 8


def test_batched_full_recipe():
    """The whole 64-problem batched workload solved in one batched call with
    the batched tile autotuner; every problem and RHS converges, and the true
    residual of sampled problems (including the largest) is confirmed with
    the oracle's own operator."""
    specs = batched_problem_specs()
    probs, bs = [], []
    for k, sp in enumerate(specs):
        P = amg.Problem.structured(sp["N"], 0.0, None, sp["s"]).setup(coarse_max=64)
        probs.append(P)
        bs.append(rhs_uniform(P.n, 16, config=4000 + k))
    B = amg.Batch(probs, [16] * len(probs))
    xs, res = B.solve([torch.from_numpy(b).to(DEV) for b in bs], tol=1e-8, tune=1)
    assert all(r.converged for r in res)
    assert max(float(np.max(r.relres)) for r in res) <= 1e-8
    largest = int(np.argmax([p.n for p in probs]))
    for p in sorted({0, 17, 41, largest}):
        h = grid.widths(specs[p]["N"], 0.0)
        x = xs[p].cpu().numpy()
        for r in (0, 7, 15):
            rr = bs[p][r] - fv.apply(h, np.ones(probs[p].n), x[r])
            assert np.linalg.norm(rr) / np.linalg.norm(bs[p][r]) <= 1.05e-8
