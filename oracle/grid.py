"""Grid nodes for the unit-cube model problem (Sec. 2.2, eq. "tanh").

ORACLE (test infrastructure only; see ``oracle/__init__.py``).
"""

from __future__ import annotations

import numpy as np


def nodes_1d(N: int, gamma: float) -> np.ndarray:
    """Face positions ``x_0..x_N`` of an ``N``-cell axis on [0, 1].

    ``gamma == 0`` gives the uniform grid ``x_i = i/N``.  Otherwise the
    hyperbolic stretching of eq. "tanh" (Sec. 2.2), shifted to 0-based
    indices: ``x_i = (1 + tanh(gamma (2 i / N - 1)) / tanh(gamma)) / 2``.
    """
    i = np.arange(N + 1, dtype=np.float64)
    if gamma == 0.0:
        x = i / N
    else:
        x = 0.5 * (1.0 + np.tanh(gamma * (2.0 * i / N - 1.0)) / np.tanh(gamma))
    x[0] = 0.0
    x[N] = 1.0
    return x


def widths_1d(N: int, gamma: float) -> np.ndarray:
    """Cell widths ``h_i = x_{i+1} - x_i`` of ``nodes_1d``.

    For even ``N`` the upper half is the exact reflection of the lower half
    (``h_{N-1-i} = h_i`` bit for bit): the tanh map is odd about the
    mid-plane, but rounding alone would not keep mirror cells identical, and
    the mirrored ordering of Sec. 2 needs them identical.
    """
    h = np.diff(nodes_1d(N, gamma))
    if N % 2 == 0:
        half = N // 2
        h[half:] = h[:half][::-1]
    return h


def widths(N, gamma: float):
    """Per-axis cell widths for a tensor grid ``N = (Nx, Ny[, Nz])``."""
    return [widths_1d(int(n), gamma) for n in N]
