"""Pins for the beta weights (oracle.quadrature).

Clenshaw-Curtis on x_k = cos(k pi/(N-1)): checked against the moment
conditions it must satisfy (exact integrals of monomials), against an
independent construction by a linear solve of the moment system, and against
symmetry.  The paper-literal Riemann weights (Sec. 4 factorised Riemann sum,
sin(theta_k) with cell width pi/(N-1)) are checked for their convergence to
int_0^pi sin = 2.
"""
import numpy as np
import pytest

from oracle import quadrature


@pytest.mark.parametrize("N", [4, 5, 8, 16, 33, 64, 256])
def test_cc_sum_and_symmetry(N):
    w = quadrature.clenshaw_curtis(N)
    assert abs(w.sum() - 2.0) < 1e-13
    assert np.allclose(w, w[::-1], atol=1e-15, rtol=0)
    assert np.all(w > 0)


@pytest.mark.parametrize("N", [4, 7, 8, 16, 32, 64])
def test_cc_exact_on_monomials(N):
    w = quadrature.clenshaw_curtis(N)
    x = np.cos(np.pi * np.arange(N) / (N - 1))
    for p in range(N):
        exact = 2.0 / (p + 1) if p % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** p) - exact) < 1e-13, p
    if N <= 8:
        # a degree past the rule's exactness is no longer integrated exactly
        p = N if N % 2 == 0 else N + 1
        assert abs(np.dot(w, x ** p) - 2.0 / (p + 1)) > 1e-6


@pytest.mark.parametrize("N", [4, 6, 9, 12])
def test_cc_matches_moment_solve(N):
    # Independent construction: interpolatory weights solve sum_k w_k T_j(x_k) = int T_j.
    x = np.cos(np.pi * np.arange(N) / (N - 1))
    V = np.polynomial.chebyshev.chebvander(x, N - 1).T      # V[j, k] = T_j(x_k)
    rhs = np.array([2.0 / (1 - j * j) if j % 2 == 0 else 0.0 for j in range(N)])
    w_ref = np.linalg.solve(V, rhs)
    assert np.allclose(quadrature.clenshaw_curtis(N), w_ref, atol=1e-13, rtol=0)


def test_riemann_literal_converges():
    # The literal weights are the trapezoidal rule for int_0^pi sin = 2 (both end
    # values vanish); its Euler-Maclaurin leading error is h^2/12 * (f'(pi) - f'(0))
    # = -pi^2 / (6 (N-1)^2).
    for N in (16, 64, 256):
        err = quadrature.riemann(N).sum() - 2.0
        lead = -np.pi ** 2 / (6 * (N - 1) ** 2)
        assert abs(err - lead) < 0.01 * abs(lead)
    w = quadrature.riemann(16)
    assert w[0] == 0.0 and abs(w[-1]) < 1e-15
