"""The V-cycle entry point that allocates nothing (marked gpu).

``amgsym_vcycle_noalloc`` serves callers that cannot let the library call
cudaMalloc (a real-time loop that cannot take the implicit device
synchronisation, or a process whose device memory belongs to another
allocator).  It runs the same kernels with the same tiles on the same inputs as
``amgsym_vcycle``, so it must give the same bits, call after call, with its
work vectors in the library's fixed 32 MiB device array, and reject problems
that do not fit.  This file is collected last so that a run stopping
at the first failure has run every other test already.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from synth import gaussian_logk  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32])
def test_vcycle_noalloc_matches_vcycle_on_consecutive_calls(prec):
    N, s = (32, 32, 24), 3
    g = gaussian_logk(N, s, seed=21, corr=3.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64)
    nrhs = 2
    C = nrhs << s
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    rng = np.random.default_rng(3)
    for call in range(2):  # two calls in a row, different inputs each time
        R = torch.from_numpy(rng.standard_normal((P.n_b, C))).to(DEV, dt)
        Z_ref = torch.empty_like(R)
        Z_new = torch.full_like(R, float("nan"))
        P.vcycle(R, Z_ref, nrhs, prec)
        code = amg.lib.amgsym_vcycle_noalloc(
            P._h, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z_new.data_ptr()), nrhs, prec, 0,
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == 0, amg.lib.amgsym_last_error().decode()
        torch.cuda.synchronize()
        a = Z_new.cpu().numpy()
        b = Z_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


def test_vcycle_noalloc_rejects_problems_beyond_the_scratch():
    # 128^3 with three symmetries: the finest level alone needs
    # 2 x 262144 x 8 x 8 bytes = 32 MiB, plus the coarse levels -> too large.
    N, s = (128, 128, 128), 3
    P = amg.Problem.structured(N, 0.0, None, s).setup()
    C = 1 << s
    R = torch.zeros((P.n_b, C), dtype=torch.float64, device=DEV)
    Z = torch.empty_like(R)
    with pytest.raises(amg.AmgsymError) as e:
        P.vcycle_noalloc(R, Z, 1, amg.PREC_FP64)
    assert e.value.name == "ERR_ARG"
    assert "33554432" in str(e.value)
    # the allocating entry point still serves it
    P.vcycle(R, Z, 1, amg.PREC_FP64)
    torch.cuda.synchronize()
