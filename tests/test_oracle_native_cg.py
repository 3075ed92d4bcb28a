"""Pins of the oracle's OpenMP conjugate gradients (``oracle/cg_omp.c``),
the CPU baseline's solver: it must run the iteration of ``oracle.solvers.cg``
(same coefficients), reach the exact solution, and give the same iterates on
any number of threads up to the rounding of the parallel dot products."""

import numpy as np
import pytest

from oracle import fv, grid, native, solvers
from synth import gaussian_logk


def _problem(N, gamma, vark, seed=3):
    g = gaussian_logk(N, 1, seed=seed, corr=2.0) if vark else None
    k = np.exp(g) if vark else np.ones(int(np.prod(N)))
    A = fv.assemble(grid.widths(N, gamma), k)
    b = np.random.default_rng(seed).uniform(-1.0, 1.0, A.shape[0])
    return A, b


def test_coefficients_equal_the_python_iteration():
    # the CG recurrence amplifies rounding from one iteration to the next
    # (the two sides sum their dot products in different orders), so compare
    # the first 20 coefficients on a problem far from converged by then
    A, b = _problem((48, 40, 32), 1.5, True)
    _, al, be = solvers.cg_sample(A, b, 20)
    _, info = native.cg(A, b, 20, 0.0)
    assert info["iters"] == 20
    assert np.max(np.abs(info["alphas"] - al) / np.abs(al)) <= 1e-10
    assert np.max(np.abs(info["betas"] - be) / np.abs(be)) <= 1e-10


def test_reaches_the_exact_solution():
    N = (16, 12, 10)
    A, b = _problem(N, 0.0, False)
    x, info = native.cg(A, b, 10000, 1e-13)
    assert info["relres"] <= 2e-13
    xo = solvers.dst_solve(N, b)
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)
    _, pinfo = solvers.cg(A, b, tol=1e-13, return_info=True)
    assert abs(info["iters"] - pinfo["iters"]) <= 2


@pytest.mark.parametrize("threads", [1, 2, 3])
def test_thread_count_changes_only_rounding(threads):
    A, b = _problem((48, 40, 32), 1.5, True, seed=5)
    x1, i1 = native.cg(A, b, 20, 0.0, threads=1)
    xt, it = native.cg(A, b, 20, 0.0, threads=threads)
    assert it["threads"] == threads
    assert np.linalg.norm(xt - x1) <= 1e-10 * np.linalg.norm(x1)


def test_lanczos_estimate_from_the_coefficients_bounds_kappa():
    # uniform grid: the condition number is the closed form's ratio
    N = (24, 20, 16)
    A, b = _problem(N, 0.0, False)
    lam = solvers.closed_form_eigenvalues(N)
    kappa = lam[-1] / lam[0]
    _, info = native.cg(A, b, 150, 0.0)
    est = solvers.lanczos_condition_estimate(info["alphas"], info["betas"])
    assert est <= kappa * (1 + 1e-8)
    assert est >= 0.9 * kappa
