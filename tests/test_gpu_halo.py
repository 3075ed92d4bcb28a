"""Halo-staged coarse-level products (marked gpu).

With ``halo_kb`` > 0 the CSR matrices below the finest level also carry a
halo-tiled form, and their products stage each tile's X rows in shared memory
before gathering.  The entry lanes, batches and fma order are those of the
CSR kernel, so a V-cycle with the halo form must give the same bits as one
without it, in every precision, at column counts whose halos fit shared
memory (8 columns) and at ones that fall back to the CSR kernel.  The halo
form runs only on matrices with enough tiles to fill the GPU (two per SM),
so the grids here are large enough for the first coarse levels to have them."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2407_05930_gb300 as amg  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _pair(N, s, **kw):
    g = gaussian_logk(N, s, seed=14, corr=3.0)
    # the CSR kernel as the comparison (sell=0): tuned solves then time the same candidates
    P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, precisions=7, halo_kb=64, sell=0, **kw)
    Q = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, precisions=7, halo_kb=0, sell=0, **kw)
    return P, Q


@pytest.mark.parametrize("nrhs", [1, 4])
@pytest.mark.parametrize("prec", [amg.PREC_FP64, amg.PREC_MIXED_FP32, amg.PREC_MIXED_BF16])
def test_vcycle_with_halo_products_is_bit_identical(nrhs, prec):
    N, s = (128, 96, 96), 3
    P, Q = _pair(N, s)
    C = nrhs << s
    dt = torch.float64 if prec == amg.PREC_FP64 else torch.float32
    R = torch.from_numpy(np.random.default_rng(5).standard_normal((P.n_b, C))).to(DEV, dt)
    Za, Zb = torch.empty_like(R), torch.empty_like(R)
    P.vcycle(R, Za, nrhs, prec)
    Q.vcycle(R, Zb, nrhs, prec)
    torch.cuda.synchronize()
    assert torch.equal(Za, Zb)


def test_halo_products_are_used_and_solves_agree():
    N, s = (128, 96, 96), 2
    P, Q = _pair(N, s)
    b = torch.from_numpy(rhs_uniform(P.n, 1, config=14)).to(DEV)
    recs = P.profile_step(b, torch.empty_like(b), 1, amg.PREC_MIXED_FP32)
    halo = [r for r in recs if r["kernel"].startswith("spmm_halo_kernel")]
    assert halo and all(r["level"] >= 0 for r in halo)
    assert any(r["role"].startswith("L1 A") for r in halo)
    assert not any(r["kernel"].startswith("spmm_halo_kernel")
                   for r in Q.profile_step(b, torch.empty_like(b), 1, amg.PREC_MIXED_FP32))
    for prec in (amg.PREC_FP64, amg.PREC_MIXED_FP32):
        xa, ia = P.solve(b, tol=1e-10, precision=prec)
        xb, ib = Q.solve(b, tol=1e-10, precision=prec)
        assert torch.equal(xa, xb) and ia.iters == ib.iters


def test_small_halo_budget_takes_shorter_tiles():
    N, s = (128, 96, 96), 2
    g = gaussian_logk(N, s, seed=15, corr=3.0)
    Q = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, halo_kb=0)
    nrhs, C = 1, 1 << s
    R = torch.from_numpy(np.random.default_rng(6).standard_normal((Q.n_b, C))).to(DEV, torch.float32)
    Zq = torch.empty_like(R)
    Q.vcycle(R, Zq, nrhs, amg.PREC_MIXED_FP32)
    for kb in (1, 4, 16):
        P = amg.Problem.structured(N, 1.5, g, s).setup(coarse_max=64, halo_kb=kb)
        Zp = torch.empty_like(R)
        P.vcycle(R, Zp, nrhs, amg.PREC_MIXED_FP32)
        torch.cuda.synchronize()
        assert torch.equal(Zp, Zq), kb
