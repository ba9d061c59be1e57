"""Pins for the Sec. 4 shifted-polynomial identities (oracle.shifted).

Every projection form is compared with <s, P_{L+r}> built from scipy's
Legendre polynomials on the Chebyshev-Lobatto beta nodes.
"""
import numpy as np
import pytest
import scipy.special as sps

from oracle import shifted

N = 64
X = np.cos(np.pi * np.arange(N) / (N - 1))


def direct(s, deg):
    return float(np.dot(s, sps.eval_legendre(deg, X)))


def test_lemma_matches_scipy():
    P = shifted.legendre_lemma(120, X)
    for l in range(121):
        assert np.max(np.abs(P[l] - sps.eval_legendre(l, X))) < 1e-12


@pytest.mark.parametrize("L,r", [(1, 1), (3, 4), (10, 17), (25, 30)])
def test_basic_projection(L, r):
    s = np.random.default_rng(L * 100 + r).standard_normal(N)
    assert abs(shifted.projection_k1(s, L, r, X) - direct(s, L + r)) < 1e-11


def test_shift_definition():
    # P_{L+r} = A_r^L P_L + B_r^L P_{L-1}, initial A_0 = 1, B_0 = 0, A_-1 = 0, B_-1 = 1
    L = 7
    A, B = shifted.shifted_AB(L, 20, X)
    for r in range(-1, 21):
        lhs = sps.eval_legendre(L + r, X)
        rhs = A[r + 1] * sps.eval_legendre(L, X) + B[r + 1] * sps.eval_legendre(L - 1, X)
        assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_composition_rule():
    # [[A_{r+s}, B_{r+s}], [A_{r+s-1}, B_{r+s-1}]] = M_s^{L+r} M_r^L
    L, r, s_ = 5, 6, 9
    def M(Lb, rr):
        A, B = shifted.shifted_AB(Lb, rr, X)
        return np.array([[A[rr + 1], B[rr + 1]], [A[rr], B[rr]]])
    lhs = M(L, r + s_)
    Ms, Mr = M(L + r, s_), M(L, r)
    rhs = np.einsum("abk,bck->ack", Ms, Mr)
    assert np.max(np.abs(lhs - rhs)) < 1e-11
    # A_r^0 = P_r, B_r^0 = 0
    A0, B0 = shifted.shifted_AB(0, 12, X)
    for rr in range(1, 13):
        assert np.max(np.abs(A0[rr + 1] - sps.eval_legendre(rr, X))) < 1e-12
        assert np.max(np.abs(B0[rr + 1])) < 1e-15


@pytest.mark.parametrize("parts", [(3, 4), (1, 1), (7, 2)])
def test_k2_example_four_terms(parts):
    L = 6
    s = np.random.default_rng(sum(parts)).standard_normal(N)
    ref = direct(s, L + sum(parts))
    assert abs(shifted.projection_split(s, L, list(parts), X) - ref) < 1e-11
    # the printed general formula coincides with the composition rule at k = 2
    assert abs(shifted.projection_printed(s, L, list(parts), X) - ref) < 1e-11


@pytest.mark.parametrize("parts", [(2, 3, 4), (1, 2, 1, 3), (4, 4, 4, 4, 4)])
def test_general_depth_composition_rule(parts):
    L = 5
    s = np.random.default_rng(len(parts)).standard_normal(N)
    ref = direct(s, L + sum(parts))
    assert abs(shifted.projection_split(s, L, list(parts), X) - ref) < 1e-10


def test_printed_general_formula_differs_for_k3():
    # Reading recorded in the design notes: as printed, only n_1 is lowered by eps_1.
    L = 5
    s = np.random.default_rng(0).standard_normal(N)
    ref = direct(s, L + 9)
    assert abs(shifted.projection_printed(s, L, [2, 3, 4], X) - ref) > 1e-6
