"""Per-launch timing of one solve step (amgsym_profile_step, marked gpu).

The profiled step must leave the problem as it found it (a solve after it
gives the same bits as a solve before it), time every launch of one PCG
iteration, and count the reduced SpMM's algorithmic bytes by the formula of
its storage: the stored diagonals, X and Y once, the interface lookups."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("prec", [amg.PREC_MIXED_FP32, amg.PREC_FP64])
def test_profile_step_records_one_iteration(prec):
    N, s = (64, 64, 48), 3
    g = gaussian_logk(N, s, seed=12, corr=4.0)
    P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64)
    b = torch.from_numpy(rhs_uniform(P.n, 1, config=12)).to(DEV)
    x1, i1 = P.solve(b, tol=1e-10, precision=prec)
    recs = P.profile_step(b, torch.empty_like(b), 1, prec)
    x2, i2 = P.solve(b, tol=1e-10, precision=prec)
    assert torch.equal(x1, x2) and i1.iters == i2.iters
    assert all(r["us"] > 0 and r["bytes"] > 0 for r in recs)
    it = [r for r in recs if r["phase"] == 1]
    roles = [r["role"] for r in it]
    assert roles[0].startswith("reduced SpMM") and roles[1].startswith("x += a p")
    assert roles[-1] == "p = z + b p"
    assert sum("dense coarsest solve" in r for r in roles) == 1
    levels = {r["level"] for r in it if r["level"] >= 0}
    assert levels == set(range(P.num_levels()))
    # the reduced SpMM's bytes: stored diagonals (FP64 or FP32 values), X = p
    # (also the dot's partner) and Y = q once, the interface lookups
    w = 8 if prec == amg.PREC_FP64 else 4
    C = P.nb
    dia = P.level_dia(0, "A")
    sz = P.sizes()
    words = (P.n_b + 31) // 32
    iface = words * 8 + (sz["n_iface_rows"] + 1) * 4 + sz["n_iface_rows"] * 4 + sz["n_iface_entries"] * (4 + w * C)
    assert dia["ndiag"] == 7
    assert it[0]["bytes"] == dia["nstored"] * P.n_b * w + 2 * C * w * P.n_b + iface
    kinds = {r["kernel"].split("<")[0] for r in recs}
    assert {"transform_fwd_kernel", "transform_bwd_kernel", "spmm_kernel", "cg_update1_kernel",
            "cg_update2_kernel", "coarse_kernel"} <= kinds
