"""GPU parity of the individual steps through the C ABI (marked gpu).

Transform (Alg. 1 first/last step, eq. "P_s"), reduced operator (eq.
"hL_splitting", fused SpMM + interface), and the V-cycle preconditioner
(symmetry and positivity), each against the FP64 oracle on seeded inputs
spanning several thread blocks with ragged tails.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from gpu_common import oracle_apply_hat, oracle_forward, oracle_hat_blocks, oracle_problem  # noqa: E402
from synth import rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [
    ((64, 64), 1, 1, 0.0, False),      # 2D 5-point, one symmetry
    ((30, 22, 18), 3, 1, 1.5, True),   # ragged 3D, three symmetries, stretched var-k
    ((20, 14, 10), 2, 3, 1.5, True),   # nrhs = 3, s = 2 -> 12 columns
    ((12, 10, 8), 0, 3, 0.0, False),   # no symmetry, odd column count
    ((16, 16, 16), 3, 4, 0.0, False),  # 32 columns
]


def _problem(N, s, gamma, vark):
    g, h, k, A = oracle_problem(N, s, gamma, vark)
    P = amg.Problem.structured(N, gamma, g, s).setup(coarse_max=64)
    return P, A


@pytest.mark.parametrize("N,s,nrhs,gamma,vark", CASES)
def test_transform_forward_backward(N, s, nrhs, gamma, vark):
    P, A = _problem(N, s, gamma, vark)
    b = rhs_uniform(P.n, nrhs, config=11)
    bt = torch.from_numpy(b).to(DEV)
    C = nrhs << s
    xh = torch.empty((P.n_b, C), dtype=torch.float64, device=DEV)
    P.transform_forward(bt, nrhs, xh)
    ref = oracle_forward(b, N, s)
    got = xh.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
    back = torch.empty_like(bt)
    P.transform_backward(xh, nrhs, back)
    assert np.max(np.abs(back.cpu().numpy() - b)) <= 1e-15 * 2 ** s


@pytest.mark.parametrize("s", [1, 2, 3])
def test_transform_integer_roundtrip_bit_exact(s):
    N = (16, 12, 10)
    P = amg.Problem.structured(N, 0.0, None, s).setup(coarse_max=64)
    rng = np.random.default_rng(s)
    b = rng.integers(-(2 ** 20), 2 ** 20, size=(2, P.n)).astype(np.float64)
    bt = torch.from_numpy(b).to(DEV)
    xh = torch.empty((P.n_b, 2 << s), dtype=torch.float64, device=DEV)
    P.transform_forward(bt, 2, xh)
    # unnormalised butterfly of integers is exact
    assert np.array_equal(xh.cpu().numpy(), oracle_forward(b, N, s).round())
    back = torch.empty_like(bt)
    P.transform_backward(xh, 2, back)
    assert np.array_equal(back.cpu().numpy(), b)


@pytest.mark.parametrize("N,s,nrhs,gamma,vark", CASES)
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_apply_reduced(N, s, nrhs, gamma, vark, prec):
    P, A = _problem(N, s, gamma, vark)
    perm, hat = oracle_hat_blocks(A, N, s)
    C = nrhs << s
    X = np.random.default_rng(5).uniform(-1, 1, (P.n_b, C))
    Yref = oracle_apply_hat(hat, X, 1 << s)
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    Xt = torch.from_numpy(X).to(DEV, dt)
    Yt = torch.empty_like(Xt)
    P.apply_reduced(Xt, Yt, nrhs, prec)
    Y = Yt.double().cpu().numpy()
    scale = np.max(np.abs(A.data)) * np.max(np.abs(X))
    tol = 1e-14 if prec == amg.PREC_FP64 else 1e-6
    assert np.max(np.abs(Y - Yref)) <= tol * scale * 8


@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_vcycle_symmetric_positive(prec):
    N, s = (32, 32, 24), 3
    g, h, k, A = oracle_problem(N, s, 1.5, True)
    P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, precisions=7)
    nrhs = 2
    C = nrhs << s
    rng = np.random.default_rng(7)
    U = rng.standard_normal((P.n_b, C))
    V = rng.standard_normal((P.n_b, C))
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    Ut, Vt = torch.from_numpy(U).to(DEV, dt), torch.from_numpy(V).to(DEV, dt)
    MU, MV = torch.empty_like(Ut), torch.empty_like(Vt)
    P.vcycle(Ut, MU, nrhs, prec)
    P.vcycle(Vt, MV, nrhs, prec)
    MU = MU.double().cpu().numpy()
    MV = MV.double().cpu().numpy()
    tol = 1e-12 if prec == amg.PREC_FP64 else 1e-5
    for c in range(C):
        a = MU[:, c] @ V[:, c]
        b = U[:, c] @ MV[:, c]
        assert abs(a - b) <= tol * (abs(a) + abs(b))
        assert MU[:, c] @ U[:, c] > 0
    # determinism: the same input gives the same bits
    MU2 = torch.empty_like(Ut)
    P.vcycle(Ut, MU2, nrhs, prec)
    assert np.array_equal(MU2.double().cpu().numpy(), MU)
