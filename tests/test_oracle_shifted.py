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


# ---------------------------------------------------------------------------
# The (m, n) analogue (Wigner-d recurrence) and the depth-k forward transform
# ---------------------------------------------------------------------------
from oracle import basis, grid as OG, transform as OT  # noqa: E402

BETA = np.pi * np.arange(N) / (N - 1)
PAIRS = [(0, 0), (2, -4), (1, 1), (-7, 3), (20, 20), (-31, 29), (62, 0), (5, -63)]


@pytest.mark.parametrize("n2,m2", PAIRS)
def test_wigner_shift_definition(n2, m2):
    """d^{L+r} = A_r^L d^L + B_r^L d^{L-1} against the independently pinned column."""
    jtop = 63 if n2 % 2 else 62
    j0, D = basis.wigner_d_column(n2, m2, BETA, jtop)
    if D.shape[0] < 3:
        pytest.skip("no shift")
    for base in (1, D.shape[0] // 2):
        A, B = shifted.wigner_shifted_AB(n2, m2, j0 + 2 * base, D.shape[0] - 1 - base, X)
        for r in range(-1, D.shape[0] - base):
            rhs = A[r + 1] * D[base] + B[r + 1] * D[base - 1]
            assert np.max(np.abs(D[base + r] - rhs)) < 1e-12


def test_wigner_shift_reduces_to_legendre():
    A, B = shifted.wigner_shifted_AB(0, 0, 14, 20, X)
    A0, B0 = shifted.shifted_AB(7, 20, X)
    assert np.max(np.abs(A - A0)) < 1e-12 and np.max(np.abs(B - B0)) < 1e-12


def test_wigner_composition_rule():
    """The 2 x 2 transfer matrices compose: shift n1 then n2 equals shift n1 + n2."""
    n2, m2, L2 = 3, -9, 11
    n1, nn2 = 5, 7
    A, B = shifted.wigner_shifted_AB(n2, m2, L2, n1 + nn2, X)
    A1, B1 = shifted.wigner_shifted_AB(n2, m2, L2, n1, X)
    A2, B2 = shifted.wigner_shifted_AB(n2, m2, L2 + 2 * n1, nn2, X)
    lhs = A[n1 + nn2 + 1]
    rhs = A2[nn2 + 1] * A1[n1 + 1] + B2[nn2 + 1] * A1[n1]
    assert np.max(np.abs(lhs - rhs)) < 1e-10 * max(1.0, np.max(np.abs(lhs)))


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("n2,m2", [(0, 0), (1, -1), (-7, 3), (20, 20), (-30, 12)])
def test_wigner_depth_projection_matches_direct(k, n2, m2):
    jtop = 63 if n2 % 2 else 62
    j0, D = basis.wigner_d_column(n2, m2, BETA, jtop)
    s = np.random.default_rng(k * 1000 + n2 * 7 + m2).standard_normal(N)
    R = D.shape[0] - 2
    b = shifted.depth_base(R, k)
    for r in range(1, R + 1):
        parts = shifted.digit_parts(r, b, k)
        assert sum(parts) == r and len(parts) == k
        got = shifted.wigner_projection(s, D[1], D[0], n2, m2, j0 + 2, parts, X)
        assert abs(got - np.dot(D[r + 1], s)) < 1e-12 * max(1.0, np.max(np.abs(D @ s)))


def test_digit_parts():
    assert shifted.depth_base(63, 1) == 64 and shifted.depth_base(63, 2) == 8 and shifted.depth_base(63, 3) == 4
    assert shifted.digit_parts(45, 4, 3) == [32, 12, 1]
    assert shifted.digit_parts(7, 8, 2) == [0, 7]


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("Nf", [8, 16])
def test_forward_depth_equals_definition(k, Nf):
    """The depth-k transform equals the plain quadrature sum (direct O(N^6) at
    N = 8, the separated form at N = 16)."""
    rng = np.random.default_rng(400 + 10 * k + Nf)
    f = rng.standard_normal((Nf, Nf, Nf)) + 1j * rng.standard_normal((Nf, Nf, Nf))
    ref = OT.forward_direct(f) if Nf == 8 else OT.forward_separable(f)
    got = shifted.forward_depth(f, k)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
