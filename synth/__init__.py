"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This module draws random numbers and nothing else of the method: no matrix
assembly, no symmetry transform, no solver arithmetic.  Both the CPU oracle
(``oracle/``) and the CUDA library's tests and benchmark take their inputs
from here, so that the two sides see bit-identical data without sharing any
of the method's code.

Recipes (all FP64, numpy ``default_rng``):

* right-hand sides: i.i.d. uniform[-1, 1] over the full grid with no
  symmetry imposed, so every decoupled block is excited; seed
  ``1000 * config + rhs`` (the paper uses "a random vector", Sec. 5);
* log-coefficient field ``g``: i.i.d. N(0, 1) on the base octant, mirrored
  to the full grid, smoothed by a separable Gaussian filter of standard
  deviation ``corr`` cells (truncated at 4 sigma, reflecting boundaries),
  re-mirrored so that the symmetry is exact bit for bit, then standardised to
  mean 0 and standard deviation ``sigma``; ``k = exp(g)`` is formed by the
  consumer;
* adjoint targets ``u_t``: i.i.d. N(0, 1), seed ``5000 + i``.

Array convention: a field on an ``N = (Nx, Ny[, Nz])`` grid is a flat FP64
vector in natural lexicographic order with x fastest, i.e. a C-ordered array
of shape ``N[::-1]`` flattened.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "CONFIGS",
    "rhs_uniform",
    "gaussian_logk",
    "u_target",
    "batched_problem_specs",
]

# Workload recipes: grid cells per axis, stretching gamma (0 = uniform),
# number of reflection symmetries s, RHS count, relative-residual tolerance,
# whether k is the smoothed random field.
CONFIGS = {
    1: dict(name="2d5pt_64x64_s1", N=(64, 64), gamma=0.0, s=1, nrhs=1, tol=1e-10, vark=False),
    2: dict(name="3d7pt_128cube_s3", N=(128, 128, 128), gamma=0.0, s=3, nrhs=4, tol=1e-10, vark=False),
    3: dict(name="3d7pt_vark_tanh_256cube_s3", N=(256, 256, 256), gamma=1.5, s=3, nrhs=1, tol=1e-8, vark=True),
    4: dict(name="batched_64x_7pt", N=None, gamma=0.0, s=None, nrhs=16, tol=1e-8, vark=False),
    5: dict(name="adjoint_vark_tanh_192cube_s3", N=(192, 192, 192), gamma=1.5, s=3, nrhs=1, tol=1e-8, vark=True),
}


def rhs_uniform(n: int, nrhs: int, config: int) -> np.ndarray:
    """``nrhs`` right-hand sides of length ``n``, uniform[-1, 1], shape (nrhs, n)."""
    out = np.empty((nrhs, n), dtype=np.float64)
    for r in range(nrhs):
        rng = np.random.default_rng(1000 * config + r)
        out[r] = rng.uniform(-1.0, 1.0, n)
    return out


def _mirror_from_base(base: np.ndarray, s: int) -> np.ndarray:
    """Tile a base-octant array (C order, axes reversed) to the full grid by
    reflecting it across the upper faces of the first ``s`` axes (x, y, z)."""
    full = base
    d = base.ndim
    for a in range(s):
        ax = d - 1 - a  # numpy axis of grid axis a
        full = np.concatenate([full, np.flip(full, axis=ax)], axis=ax)
    return full


def gaussian_logk(N, s: int, seed: int, corr: float = 8.0, sigma: float = 1.0) -> np.ndarray:
    """Mirror-symmetric smoothed Gaussian field ``g`` on the full grid (flat, x fastest).

    The field is exactly symmetric under the ``s`` reflections: the value at
    a cell equals, bit for bit, the value at each of its mirror images.
    """
    from scipy.ndimage import gaussian_filter

    N = tuple(int(v) for v in N)
    d = len(N)
    shape_full = N[::-1]
    base_shape = list(shape_full)
    for a in range(s):
        if N[a] % 2:
            raise ValueError("mirrored axes need an even number of cells")
        base_shape[d - 1 - a] //= 2
    rng = np.random.default_rng(seed)
    base = rng.standard_normal(size=tuple(base_shape))
    full = _mirror_from_base(base, s)
    sm = gaussian_filter(full, sigma=corr, mode="reflect", truncate=4.0)
    # Restore exact symmetry: keep the base octant, re-mirror it.
    sl = tuple(slice(0, b) for b in base_shape)
    sm = _mirror_from_base(np.ascontiguousarray(sm[sl]), s)
    sm = (sm - sm.mean()) / sm.std() * sigma
    return np.ascontiguousarray(sm).reshape(-1)


def u_target(n: int, i: int = 0) -> np.ndarray:
    """Adjoint target field, i.i.d. N(0, 1), seed ``5000 + i``."""
    return np.random.default_rng(5000 + i).standard_normal(n)


def batched_problem_specs(count: int = 64, nmin: int = 32, nmax: int = 160, seed0: int = 7000):
    """Sizes and symmetry counts of the batched workload: cube edge ``N``
    uniform over the even integers in [nmin, nmax], ``s`` uniform in {1, 2, 3};
    problem ``p`` uses seed ``seed0 + p``."""
    specs = []
    evens = np.arange(nmin, nmax + 1, 2)
    for p in range(count):
        rng = np.random.default_rng(seed0 + p)
        N = int(rng.choice(evens))
        s = int(rng.integers(1, 4))
        specs.append(dict(N=(N, N, N), s=s, seed=seed0 + p))
    return specs
