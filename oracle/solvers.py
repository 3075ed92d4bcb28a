"""Reference solves of ``A x = b`` (ORACLE; test infrastructure only).

The symmetry-reduced method of Alg. 1 ("symsolver") reaches, up to rounding,
the solution of the full system, so the oracle solves the full system by
definition:

* ``dense_solve``: Cholesky factorisation of the assembled matrix (small n);
* ``cg``: unpreconditioned conjugate gradients in FP64 (the paper's outer
  Krylov method is PCG, Sec. 5) on the full operator;
* ``dst_solve``: exact solve for uniform-grid, unit-coefficient Dirichlet
  problems through the separable sine basis (closed form below);
* ``closed_form_eigenvalues``: the spectrum of that uniform-grid operator.

Closed form: on a uniform axis of ``N`` cells the 1D operator with the
Dirichlet value on the boundary faces is ``tridiag(-1, 2, -1)`` with corner
entries 3; its eigenpairs are ``4 sin^2(m pi / (2N))`` and
``sin(m pi (j + 1/2) / N)``, ``m = 1..N``.  The d-D operator of
``oracle.fv`` is the Kronecker sum of these, axis ``a`` weighted by
``c_a = (prod_{b != a} h_b) / h_a``.
"""

from __future__ import annotations

import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def dense_solve(A, b: np.ndarray) -> np.ndarray:
    """Cholesky solve with the dense matrix (``n`` up to a few thousand)."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    c = sla.cho_factor(Ad, lower=True)
    return sla.cho_solve(c, b)


def cg(A, b: np.ndarray, tol: float = 1e-13, maxit: int = 200000, x0=None, return_info=False):
    """Plain conjugate gradients on ``A x = b`` (FP64).

    Stops when the recurrence residual satisfies ``||r|| <= tol ||b||`` and
    then confirms with the true residual ``b - A x``; if that has drifted
    above the tolerance, the iteration restarts from the current ``x``.
    """
    b = np.asarray(b, dtype=np.float64)
    bn = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if bn == 0.0:
        return (x, dict(iters=0, relres=0.0)) if return_info else x
    it_total = 0
    for _restart in range(4):
        r = b - A @ x
        p = r.copy()
        rr = float(r @ r)
        while it_total < maxit and np.sqrt(rr) > tol * bn:
            q = A @ p
            alpha = rr / float(p @ q)
            x += alpha * p
            r -= alpha * q
            rr_new = float(r @ r)
            p *= rr_new / rr
            p += r
            rr = rr_new
            it_total += 1
        true_rel = float(np.linalg.norm(b - A @ x)) / bn
        if true_rel <= tol or it_total >= maxit:
            break
    info = dict(iters=it_total, relres=true_rel)
    return (x, info) if return_info else x


def cg_sample(A, b: np.ndarray, iters: int):
    """Run ``iters`` iterations of ``cg``'s loop body from x = 0 and return
    (seconds per iteration, alphas, betas).  Used to time the oracle on a
    bounded sample of a large workload; the CG coefficients define the Lanczos
    tridiagonal whose extreme Ritz values bound the spectrum from inside."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    alphas, betas = [], []
    t0 = time.perf_counter()
    for _ in range(iters):
        q = A @ p
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr
        p *= beta
        p += r
        rr = rr_new
        alphas.append(alpha)
        betas.append(beta)
    return (time.perf_counter() - t0) / iters, alphas, betas


def lanczos_condition_estimate(alphas, betas) -> float:
    """``theta_max / theta_min`` of the CG-Lanczos tridiagonal (a lower bound
    on the condition number of the matrix CG ran on)."""
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


def _axis_weights(N):
    """``c_a = (prod_{b != a} h_b) / h_a`` for a uniform grid on the unit cube."""
    h = [1.0 / n for n in N]
    c = []
    for a in range(len(N)):
        area = 1.0
        for b in range(len(N)):
            if b != a:
                area *= h[b]
        c.append(area / h[a])
    return c


def closed_form_eigenvalues(N, bc: str = "dirichlet") -> np.ndarray:
    """Sorted spectrum of the uniform unit-coefficient operator.  Dirichlet:
    modes m = 1..N per axis; Neumann: the 1D operator is tridiag(-1, 2, -1)
    with corner entries 1, eigenpairs 4 sin^2(m pi / (2N)) and
    cos(m pi (j + 1/2) / N), m = 0..N-1 (m = 0 the constant, eigenvalue 0)."""
    N = tuple(int(v) for v in N)
    c = _axis_weights(N)
    lam = np.zeros([1] * len(N))
    for a, n in enumerate(N):
        m = np.arange(1, n + 1, dtype=np.float64) if bc == "dirichlet" else np.arange(n, dtype=np.float64)
        l1 = c[a] * 4.0 * np.sin(m * np.pi / (2.0 * n)) ** 2
        shape = [1] * len(N)
        shape[a] = n
        lam = lam + l1.reshape(shape)
    return np.sort(lam.reshape(-1))


def _sine_basis(n: int) -> np.ndarray:
    """Orthonormal DST-II basis ``S[m-1, j] = c_m sin(m pi (j + 1/2) / n)``."""
    m = np.arange(1, n + 1, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    S = np.sin(m * np.pi * (j + 0.5) / n)
    S *= np.sqrt(2.0 / n)
    S[-1] *= np.sqrt(0.5)  # m = n: sin(pi (j + 1/2)) = (-1)^j has norm^2 = n
    return S


def dst_solve(N, b: np.ndarray) -> np.ndarray:
    """Exact solve of the uniform unit-coefficient Dirichlet problem: transform
    ``b`` to the separable sine basis, divide by the eigenvalues, transform back.
    ``b`` may be a single vector or a stack ``(nrhs, n)``."""
    N = tuple(int(v) for v in N)
    d = len(N)
    c = _axis_weights(N)
    b = np.asarray(b, dtype=np.float64)
    single = b.ndim == 1
    B = b.reshape((-1,) + N[::-1])
    lam = np.zeros([1] * d)
    for a, n in enumerate(N):
        m = np.arange(1, n + 1, dtype=np.float64)
        shape = [1] * d
        shape[d - 1 - a] = n
        lam = lam + (c[a] * 4.0 * np.sin(m * np.pi / (2.0 * n)) ** 2).reshape(shape)
    out = np.empty_like(B)
    for r in range(B.shape[0]):
        U = B[r]
        for a, n in enumerate(N):
            U = np.moveaxis(np.tensordot(_sine_basis(n), U, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        U = U / lam
        for a, n in enumerate(N):
            U = np.moveaxis(np.tensordot(_sine_basis(n).T, U, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        out[r] = U
    out = out.reshape(B.shape[0], -1)
    return out[0] if single else out


def _cosine_basis(n: int) -> np.ndarray:
    """Orthonormal DCT-II basis ``C[m, j] = c_m cos(m pi (j + 1/2) / n)``,
    ``m = 0..n-1``: the eigenvectors of the 1D Neumann operator."""
    m = np.arange(n, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    Cb = np.cos(m * np.pi * (j + 0.5) / n) * np.sqrt(2.0 / n)
    Cb[0] = np.sqrt(1.0 / n)
    return Cb


def neumann_dct_solve(N, b: np.ndarray) -> np.ndarray:
    """Minimum-norm solution of the uniform unit-coefficient Neumann problem
    (the paper's model problem, Sec. 2.2, on a uniform grid): transform ``b``
    to the separable cosine basis, divide by the eigenvalues, drop the
    constant mode (eigenvalue 0; a compatible ``b`` has none), transform back.
    The result has zero mean.  ``b``: one vector or a stack ``(nrhs, n)``."""
    N = tuple(int(v) for v in N)
    d = len(N)
    c = _axis_weights(N)
    b = np.asarray(b, dtype=np.float64)
    single = b.ndim == 1
    B = b.reshape((-1,) + N[::-1])
    lam = np.zeros([1] * d)
    for a, n in enumerate(N):
        m = np.arange(n, dtype=np.float64)
        shape = [1] * d
        shape[d - 1 - a] = n
        lam = lam + (c[a] * 4.0 * np.sin(m * np.pi / (2.0 * n)) ** 2).reshape(shape)
    inv = np.zeros_like(lam)
    nz = lam > 0.0
    inv[nz] = 1.0 / lam[nz]
    out = np.empty_like(B)
    for r in range(B.shape[0]):
        U = B[r]
        for a, n in enumerate(N):
            U = np.moveaxis(np.tensordot(_cosine_basis(n), U, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        U = U * inv
        for a, n in enumerate(N):
            U = np.moveaxis(np.tensordot(_cosine_basis(n).T, U, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        out[r] = U
    out = out.reshape(B.shape[0], -1)
    return out[0] if single else out


def min_norm_solve(A, b: np.ndarray) -> np.ndarray:
    """Minimum-norm solution of a singular consistent symmetric system by the
    dense eigendecomposition (eigenvalues below 1e-12 of the largest treated
    as zero): the reference for the Neumann problem at small ``n``."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    w, V = np.linalg.eigh(Ad)
    keep = w > 1e-12 * w[-1]
    return V[:, keep] @ ((V[:, keep].T @ b) / w[keep][:, None] if np.ndim(b) == 2 else (V[:, keep].T @ b) / w[keep])
