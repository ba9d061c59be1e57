"""Sampling grid and packed coefficient layout (oracle side).

Sec. 4, Definition of the sampling grid: N nodes per Euler angle,
phi_j1, psi_j2 starting at -pi, theta_k = k*pi/(N-1), k = 0..N-1.

Reading of the phi/psi spacing: the paper prints 2*pi/(N-1), which places the
last node on +pi, a duplicate of the first (-pi) for a periodic variable.  The
default here is the periodic spacing 2*pi/N (N distinct nodes starting at
-pi); ``literal=True`` gives the printed spacing.  Every oracle routine takes
the node arrays explicitly, so either grid can be analysed.

Naming: alpha = phi (first Euler angle, index j1), beta = theta (index k),
gamma = psi (index j2).  A sampled function is an array f[j1, k, j2].
"""
from __future__ import annotations

import numpy as np


def alpha_nodes(N: int, literal: bool = False) -> np.ndarray:
    """phi_j = -pi + j * h, h = 2*pi/N (default) or 2*pi/(N-1) (literal)."""
    h = 2.0 * np.pi / ((N - 1) if literal else N)
    return -np.pi + h * np.arange(N)


def gamma_nodes(N: int, literal: bool = False, full: bool = False) -> np.ndarray:
    """psi_j, same rule as phi_j (Sec. 4, sampling grid).

    full=True: the full-group grid, psi over [-2 pi, 2 pi) with 2N nodes of the
    same spacing 2 pi/N (psi_j = -2 pi + j * 2 pi/N, j = 0..2N-1).  phi in
    [-pi, pi) and psi in [-2 pi, 2 pi) cover SU(2) once, so integer and
    half-integer l are orthogonal there (the paper's domain covers half of it).
    """
    if full:
        if literal:
            raise ValueError("the full-group grid has the periodic spacing only")
        return -2.0 * np.pi + (2.0 * np.pi / N) * np.arange(2 * N)
    return alpha_nodes(N, literal)


def beta_nodes(N: int) -> np.ndarray:
    """theta_k = k*pi/(N-1), k = 0..N-1 (Sec. 4, sampling grid)."""
    return np.pi * np.arange(N) / (N - 1)


# ---------------------------------------------------------------------------
# Packed coefficient layout.  Indices are carried doubled (j = 2l, a = 2m,
# b = 2n) so that half-integers stay exact integers.
# ---------------------------------------------------------------------------

def num_coeffs(N: int) -> int:
    """sum_{j=0}^{N-1} (j+1)^2 = N(N+1)(2N+1)/6."""
    return N * (N + 1) * (2 * N + 1) // 6


def block_offset(j: int) -> int:
    """Start of block j = 2l: sum_{i<j} (i+1)^2."""
    return j * (j + 1) * (2 * j + 1) // 6


def coeff_index(j: int, a: int, b: int) -> int:
    """Packed index of f^(l)_{mn} with j=2l, a=2m, b=2n: row m+l, column n+l."""
    r = (a + j) // 2
    c = (b + j) // 2
    return block_offset(j) + r * (j + 1) + c


def block(coeffs: np.ndarray, j: int) -> np.ndarray:
    """View of block j as a (j+1) x (j+1) matrix, rows m = -l..l, columns n."""
    o = block_offset(j)
    return coeffs[..., o:o + (j + 1) ** 2].reshape(coeffs.shape[:-1] + (j + 1, j + 1))


def half_range(j: int) -> np.ndarray:
    """Doubled indices a = 2m for m = -l, ..., l (j = 2l)."""
    return np.arange(-j, j + 1, 2)
