"""Weights for the beta (theta) sum of the discretised analysis integral.

Sec. 4 writes the analysis integral with measure sin(theta) d theta and
replaces it by a Riemann sum with weight sin(theta_k) (factorised Riemann-sum
Proposition).  With x = cos(theta), sin(theta) d theta = dx on [-1, 1], so the
beta sum is a quadrature rule on the nodes x_k = cos(k*pi/(N-1)), which are the
Chebyshev-Lobatto points.

* ``clenshaw_curtis`` (default reading): the interpolatory rule on those nodes
  (Clenshaw & Curtis, 1960).  It integrates every polynomial of degree <= N-1
  exactly, which covers all products d^l_{nm} d^{l'}_{nm} with l, l' <= (N-1)/2
  in one sector, so analysis after synthesis is exact there.
* ``riemann`` (paper-literal): w_k = sin(theta_k) * pi/(N-1), the printed
  weight with the cell width restored.
"""
from __future__ import annotations

import numpy as np


def clenshaw_curtis(N: int) -> np.ndarray:
    """Clenshaw-Curtis weights for int_{-1}^{1} g(x) dx on x_k = cos(k*pi/n), n = N-1.

    Written from the construction of the rule: interpolate g at the n+1 nodes
    by p(x) = sum''_{j=0}^{n} a_j T_j(x) with a_j = (2/n) sum''_k g_k cos(j k pi/n)
    (sum'' halves the first and last terms), then integrate term by term using
    int T_j = 2/(1 - j^2) for even j and 0 for odd j.  Collecting the factor of
    g_k gives w_k = (2/n) h_k sum''_{j even} 2/(1-j^2) cos(j k pi/n), h_0 = h_n = 1/2.
    """
    n = N - 1
    if n < 1:
        raise ValueError("need at least two nodes")
    w = np.zeros(N)
    for k in range(N):
        s = 0.0
        for j in range(0, n + 1, 2):
            I_j = 2.0 / (1.0 - j * j)
            hj = 0.5 if (j == 0 or j == n) else 1.0
            s += hj * I_j * np.cos(j * k * np.pi / n)
        hk = 0.5 if (k == 0 or k == n) else 1.0
        w[k] = (2.0 / n) * hk * s
    return w


def riemann(N: int) -> np.ndarray:
    """Paper-literal weights sin(theta_k) * pi/(N-1) (Sec. 4, Riemann sum)."""
    theta = np.pi * np.arange(N) / (N - 1)
    return np.sin(theta) * (np.pi / (N - 1))


def weights(N: int, kind: str = "cc") -> np.ndarray:
    if kind == "cc":
        return clenshaw_curtis(N)
    if kind == "riemann":
        return riemann(N)
    raise ValueError(kind)
