"""Seeded synthetic inputs for the SU(2) Fourier transform workloads.

This module is shared by the FP64 oracle harness, the tests and the benchmark.
It holds random draws only: coefficient vectors in packed order, grid noise and
ragged bandwidth lists.  It contains none of the transform's arithmetic (no
basis functions, no quadrature, no DFTs); the band-limited grids themselves are
synthesised by whichever side consumes these coefficients.

Packed coefficient order: blocks j = 2l = 0, 1, ..., N-1; inside a block the
(2l+1) x (2l+1) matrix f^(l)_{mn} is stored row-major with row m + l and
column n + l, so a block starts at j(j+1)(2j+1)/6 and the whole vector has
N(N+1)(2N+1)/6 entries.  Draws are made in exactly that order.

Complex Gaussian CN(0, s2): real and imaginary parts independent N(0, s2/2),
so that E|c|^2 = s2.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "num_coeffs",
    "packed_two_l",
    "variance_profile",
    "draw_coeffs",
    "draw_grid_noise",
    "draw_ragged_bandwidths",
    "draw_grid_gaussian",
]


def num_coeffs(N: int) -> int:
    """Number of packed coefficients for bandwidth N (2l = 0..N-1)."""
    return N * (N + 1) * (2 * N + 1) // 6


def packed_two_l(N: int) -> np.ndarray:
    """2l for every packed coefficient, in packed order (int64)."""
    return np.concatenate([np.full((j + 1) ** 2, j, dtype=np.int64) for j in range(N)])


def variance_profile(N: int, kind: str) -> np.ndarray:
    """Per-coefficient variance s2(l) in packed order.

    kind: "flat" -> 1;  "inv1" -> (1+l)^-1;  "inv2" -> (1+l)^-2.
    """
    l = packed_two_l(N) / 2.0
    if kind == "flat":
        return np.ones_like(l)
    if kind == "inv1":
        return 1.0 / (1.0 + l)
    if kind == "inv2":
        return 1.0 / (1.0 + l) ** 2
    raise ValueError(f"unknown variance profile {kind!r}")


def draw_coeffs(N: int, rng: np.random.Generator, kind: str = "flat") -> np.ndarray:
    """CN(0, s2(l)) coefficients for one function, complex128, packed order.

    One (C, 2) standard-normal draw (Re then Im per element), scaled by
    sqrt(s2/2).
    """
    C = num_coeffs(N)
    z = rng.standard_normal((C, 2))
    s = np.sqrt(variance_profile(N, kind) / 2.0)
    return (z[:, 0] * s) + 1j * (z[:, 1] * s)


def draw_grid_noise(shape, var: float, rng: np.random.Generator) -> np.ndarray:
    """Pointwise complex noise: Re and Im independently N(0, var)."""
    z = rng.standard_normal(tuple(shape) + (2,))
    sd = np.sqrt(var)
    return z[..., 0] * sd + 1j * (z[..., 1] * sd)


def draw_grid_gaussian(shape, rng: np.random.Generator) -> np.ndarray:
    """i.i.d. CN(0, 1) samples on a grid (not band-limited)."""
    z = rng.standard_normal(tuple(shape) + (2,))
    return (z[..., 0] + 1j * z[..., 1]) * np.sqrt(0.5)


def draw_ragged_bandwidths(count: int, choices, rng: np.random.Generator) -> np.ndarray:
    """Uniform draw of `count` bandwidths from `choices` (int64)."""
    return rng.choice(np.asarray(choices, dtype=np.int64), size=count)
