"""Setup steps on the device (marked gpu): the smoother damping's
lambda_max(G A G^T) of every level (opts.lambda_device) follows the host
estimator's steps on the uploaded matrices, so it agrees with the host's
estimate to rounding, and the solves agree."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("N,s", [((48, 40, 32), 2), ((64, 64, 64), 3)])
def test_device_lambda_max_matches_the_host_estimate(N, s):
    g = gaussian_logk(N, s, seed=61, corr=3.0)
    P1 = amg.Problem.structured(N, 1.5, g, s).setup(lambda_device=1)
    P0 = amg.Problem.structured(N, 1.5, g, s).setup(lambda_device=0)
    H = amg.Problem.structured(N, 1.5, g, s).setup(host_only=1)
    assert P1.num_levels() == P0.num_levels() == H.num_levels() >= 3
    for l in range(P1.num_levels() - 1):
        w1, w0, wh = (Q.level_info(l)["omega"] for Q in (P1, P0, H))
        assert w0 == wh
        assert abs(w1 - w0) <= 1e-9 * w0, (l, w1, w0)
    b = torch.from_numpy(rhs_uniform(P1.n, 1, config=62)).to(DEV)
    x1, i1 = P1.solve(b, tol=1e-10, tune=0)
    x0, i0 = P0.solve(b, tol=1e-10, tune=0)
    assert i1.converged and abs(i1.iters - i0.iters) <= 1
    assert (x1 - x0).norm() <= 1e-8 * x0.norm()
