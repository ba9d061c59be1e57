"""Pins for the basis functions of the oracle (oracle.basis).

Each check ties the oracle to something outside itself:
* the Sec. 3 Theorem at l = 1/2, where the derivative definition must return
  the entries of u itself (worked by hand from the definition);
* the Sec. 3 Rodrigues-type formula in exact arithmetic (sympy) against both
  the u-polynomial form and the recurrence;
* textbook closed forms of d^{1/2} and d^1;
* scipy's Legendre and Jacobi polynomials (the m = n = 0 case is the Sec. 4
  Lemma; general (n, m) through the standard Jacobi form of d);
* invariants: d(0) = identity, d(pi) = signed anti-identity, orthogonality of
  d^l(beta), the group law d(b1 + b2) = d(b1) d(b2), and the beta
  orthogonality under the Clenshaw-Curtis weights (Sec. 3 orthonormality
  relation, beta part).
* stored exact values in tests/golden/ (written from the Rodrigues formula by
  tests/golden/make_golden.py).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sps

from oracle import basis, quadrature

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def d_val(l2, n2, m2, beta):
    j0, D = basis.wigner_d_column(n2, m2, np.atleast_1d(np.asarray(beta, float)), l2)
    return D[(l2 - j0) // 2]


def test_half_spin_is_u_itself():
    # Sec. 3 Theorem at l = 1/2: t_{-1/2,-1/2} = a, t_{-1/2,1/2} = b,
    # t_{1/2,-1/2} = c, t_{1/2,1/2} = d (by differentiating the definition once).
    rng = np.random.default_rng(0)
    ph, th, ps = rng.uniform(-np.pi, np.pi), rng.uniform(0, np.pi), rng.uniform(-np.pi, np.pi)
    a, b, c, d = basis.u_entries(ph, th, ps)
    assert np.isclose(basis.t_from_u(1, -1, -1, a, b, c, d), a, atol=1e-15)
    assert np.isclose(basis.t_from_u(1, -1, 1, a, b, c, d), b, atol=1e-15)
    assert np.isclose(basis.t_from_u(1, 1, -1, a, b, c, d), c, atol=1e-15)
    assert np.isclose(basis.t_from_u(1, 1, 1, a, b, c, d), d, atol=1e-15)
    # and u is special unitary
    U = np.array([[a, b], [c, d]])
    assert np.allclose(U @ U.conj().T, np.eye(2), atol=1e-15)
    assert np.isclose(np.linalg.det(U), 1.0, atol=1e-15)


def test_u_form_equals_rodrigues_form():
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(1)
    ph, th, ps = rng.uniform(-np.pi, np.pi), rng.uniform(0.1, 3.0), rng.uniform(-np.pi, np.pi)
    a, b, c, d = basis.u_entries(ph, th, ps)
    for j in range(0, 5):
        for m2 in range(-j, j + 1, 2):
            for n2 in range(-j, j + 1, 2):
                l, m, n = sp.Rational(j, 2), sp.Rational(m2, 2), sp.Rational(n2, 2)
                P = complex(sp.N(basis.P_rodrigues_exact(l, m, n, sp.cos(sp.Float(th, 30))), 25))
                t_rod = P * np.exp(-1j * (m2 / 2 * ph + n2 / 2 * ps))
                t_u = basis.t_from_u(j, m2, n2, a, b, c, d)
                assert abs(t_u - t_rod) < 1e-13, (j, m2, n2)


def test_recurrence_matches_rodrigues_exact():
    sp = pytest.importorskip("sympy")
    # P^l_{mn}(cos b) = i^{n-m} d^l_{mn}(b); compare with the recurrence for l <= 3.5
    for beta in (0.37, 1.9, 2.8):
        xs = sp.cos(sp.Float(beta, 30))
        for j in range(0, 8):
            for m2 in range(-j, j + 1, 2):
                for n2 in range(-j, j + 1, 2):
                    l, m, n = sp.Rational(j, 2), sp.Rational(m2, 2), sp.Rational(n2, 2)
                    P = complex(sp.N(basis.P_rodrigues_exact(l, m, n, xs), 25))
                    dv = d_val(j, m2, n2, beta)[0]            # first index m, second n
                    assert abs(P - basis.i_pow((n2 - m2) // 2) * dv) < 1e-13, (j, m2, n2)


def test_golden_exact_values():
    with open(os.path.join(GOLDEN, "wigner_exact.json")) as fh:
        g = json.load(fh)
    beta = g["beta"]
    for rec in g["values"]:
        j, a2, b2 = rec["two_l"], rec["two_first"], rec["two_second"]
        assert abs(d_val(j, a2, b2, beta)[0] - float(rec["d"])) < 1e-14, rec


def test_closed_forms_spin_half_and_one():
    for b in np.linspace(0, np.pi, 7):
        c2, s2 = np.cos(b / 2), np.sin(b / 2)
        half = {(1, 1): c2, (1, -1): -s2, (-1, 1): s2, (-1, -1): c2}
        for (n2, m2), v in half.items():
            assert abs(d_val(1, n2, m2, b)[0] - v) < 1e-15
        cb, sb = np.cos(b), np.sin(b)
        one = {(2, 2): (1 + cb) / 2, (2, 0): -sb / np.sqrt(2), (2, -2): (1 - cb) / 2,
               (0, 2): sb / np.sqrt(2), (0, 0): cb, (0, -2): -sb / np.sqrt(2),
               (-2, 2): (1 - cb) / 2, (-2, 0): sb / np.sqrt(2), (-2, -2): (1 + cb) / 2}
        for (n2, m2), v in one.items():
            assert abs(d_val(2, n2, m2, b)[0] - v) < 1e-15


@pytest.mark.parametrize("j", [0, 1, 2, 7, 15, 40, 127])
def test_poles(j):
    for n2 in range(-j, j + 1, 2):
        for m2 in range(-j, j + 1, 2):
            v0 = d_val(j, n2, m2, 0.0)[0]
            vpi = d_val(j, n2, m2, np.pi)[0]
            assert abs(v0 - (1.0 if n2 == m2 else 0.0)) < 1e-12
            exp_pi = ((-1.0) ** ((j - m2) // 2)) if n2 == -m2 else 0.0
            assert abs(vpi - exp_pi) < 1e-12


def test_legendre_special_case_matches_scipy():
    beta = np.linspace(0, np.pi, 101)
    j0, D = basis.wigner_d_column(0, 0, beta, 400)
    for l in range(0, 201):
        assert np.max(np.abs(D[l] - sps.eval_legendre(l, np.cos(beta)))) < 1e-12


def _jacobi_form(l2, n2, m2, beta):
    """Textbook Jacobi form of d^j_{m'm} (first index m' = n)."""
    j, mp, m = l2 / 2, n2 / 2, m2 / 2
    cands = [(j + m, mp - m, mp - m), (j - m, m - mp, 0), (j + mp, m - mp, 0), (j - mp, mp - m, mp - m)]
    k, a, lam = min(cands, key=lambda t: t[0])
    k, a, lam = int(round(k)), int(round(a)), int(round(lam))
    bb = int(round(2 * j - 2 * k - a))
    pref = (-1.0) ** lam * math.sqrt(math.comb(int(round(2 * j - k)), k + a) / math.comb(k + bb, bb))
    return pref * np.sin(beta / 2) ** a * np.cos(beta / 2) ** bb * sps.eval_jacobi(k, a, bb, np.cos(beta))


@pytest.mark.parametrize("j", [3, 8, 21, 40])
def test_general_pairs_match_scipy_jacobi(j):
    beta = np.linspace(0.05, np.pi - 0.05, 23)
    for n2 in range(-j, j + 1, 2):
        for m2 in range(-j, j + 1, 2):
            got = d_val(j, n2, m2, beta)
            ref = _jacobi_form(j, n2, m2, beta)
            assert np.max(np.abs(got - ref)) < 1e-11, (j, n2, m2)


@pytest.mark.parametrize("j", [5, 16, 41])
def test_orthogonal_matrix_and_group_law(j):
    b1, b2 = 0.61, 1.37
    D1 = basis.wigner_d_matrix(j, b1)
    D2 = basis.wigner_d_matrix(j, b2)
    D12 = basis.wigner_d_matrix(j, b1 + b2)
    assert np.allclose(D1 @ D1.T, np.eye(j + 1), atol=1e-12)
    assert np.allclose(D1 @ D2, D12, atol=1e-12)


@pytest.mark.parametrize("j", [255, 511])
def test_large_l_unitarity_of_rows(j):
    # sum_n d^l_{nm}(b)^2 = 1 for fixed m at large l (detects any lost or wrong term)
    beta = np.array([1e-3, 0.01233, 0.4, 1.5707, 2.9, np.pi - 0.01233])
    for m2 in (-j, -j + 2, -1 if j % 2 else 0, j // 3 * 2 + (j % 2), j):
        tot = np.zeros(beta.size)
        for n2 in range(-j, j + 1, 2):
            tot += d_val(j, n2, m2, beta) ** 2
        assert np.max(np.abs(tot - 1.0)) < 1e-11, m2


@pytest.mark.parametrize("N", [8, 16, 32])
def test_beta_orthogonality_cc(N):
    # Sec. 3 orthonormality <t^l_{nm}, t^l'_{nm}> = delta/(2l+1): beta part with the
    # 1/2 from (1/(8 pi^2)) * (2 pi)^2 gives sum_k w_k d^l d^l' = 2 delta/(2l+1).
    w = quadrature.clenshaw_curtis(N)
    beta = np.pi * np.arange(N) / (N - 1)
    for par in (0, 1):
        top = N - 1 if (N - 1) % 2 == par else N - 2
        for n2 in range(-top, top + 1, 2):
            for m2 in range(-top, top + 1, 2):
                j0, D = basis.wigner_d_column(n2, m2, beta, top)
                G = (D * w) @ D.T
                js = j0 + 2 * np.arange(D.shape[0])
                assert np.allclose(G, np.diag(2.0 / (js + 1)), atol=1e-13)


def test_symmetries():
    # d^l_{nm} = (-1)^{n-m} d^l_{mn} = d^l_{-m,-n}
    beta = np.linspace(0, np.pi, 9)
    for j in (4, 9, 30):
        for n2 in range(-j, j + 1, 2):
            for m2 in range(-j, j + 1, 2):
                v = d_val(j, n2, m2, beta)
                assert np.allclose(v, (-1.0) ** ((n2 - m2) // 2) * d_val(j, m2, n2, beta), atol=1e-13)
                assert np.allclose(v, d_val(j, -m2, -n2, beta), atol=1e-13)
