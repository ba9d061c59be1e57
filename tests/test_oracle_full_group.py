"""Pins of the oracle's full-group grid (psi over [-2 pi, 2 pi), 2N nodes,
prefactor 1/(4N^2)): two independent evaluations agree; band-limited functions
mixing both sectors are recovered exactly (the property the half domain lacks);
integer-l functions give the half-grid coefficients; half-integer-l functions
are antiperiodic in psi with period 2 pi; adjoint identity; Plancherel."""
import numpy as np
import pytest

import su2inputs as I
from oracle import grid as G
from oracle import transform as T


def _rand_grid(N, rng, full=True):
    shape = (N, N, 2 * N if full else N)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("N", [4, 8])
def test_direct_equals_separable_full(N):
    rng = np.random.default_rng(100 + N)
    f = _rand_grid(N, rng)
    a = T.forward_direct(f, full=True)
    b = T.forward_separable(f, full=True)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_full_grid_nodes_and_prefactor():
    N = 8
    ga = G.gamma_nodes(N, full=True)
    assert ga.shape == (2 * N,)
    assert ga[0] == -2 * np.pi and np.allclose(np.diff(ga), 2 * np.pi / N)
    assert np.isclose(T._prefactor(N, False, True), 1.0 / (4 * N * N))


@pytest.mark.parametrize("N", [4, 8, 16])
def test_mixed_sector_exact_recovery(N):
    """forward(inverse(c)) = c for coefficients in both sectors at once."""
    rng = np.random.default_rng(200 + N)
    c = I.draw_coeffs(N, rng)
    f = T.inverse_separable(c, N, full=True)
    back = T.forward_separable(f, full=True)
    assert np.max(np.abs(back - c)) < 1e-12 * np.max(np.abs(c))


def test_mixed_recovery_fails_on_half_domain():
    """The same mixed coefficients are not recovered on the paper's domain."""
    N = 8
    rng = np.random.default_rng(300)
    c = I.draw_coeffs(N, rng)
    f = T.inverse_separable(c, N)
    back = T.forward_separable(f)
    assert np.max(np.abs(back - c)) > 1e-3 * np.max(np.abs(c))


def test_integer_sector_matches_half_grid():
    N = 8
    rng = np.random.default_rng(400)
    c = I.draw_coeffs(N, rng)
    two_l = I.packed_two_l(N)
    c[two_l % 2 == 1] = 0
    f_full = T.inverse_separable(c, N, full=True)
    f_half = T.inverse_separable(c, N)
    # psi_half[j] = -pi + 2 pi j/N = psi_full[j + N/2]; integer l: 2 pi periodic in psi
    assert np.max(np.abs(f_full[:, :, N // 2:N // 2 + N] - f_half)) < 1e-12 * np.max(np.abs(f_half))
    assert np.max(np.abs(f_full[:, :, N:] - f_full[:, :, :N])) < 1e-12 * np.max(np.abs(f_half))
    full = T.forward_separable(f_full, full=True)
    half = T.forward_separable(f_half)
    ints = two_l % 2 == 0
    assert np.max(np.abs(full[ints] - half[ints])) < 1e-12 * np.max(np.abs(c))
    assert np.max(np.abs(full[~ints])) < 1e-12 * np.max(np.abs(c))


def test_half_integer_sector_antiperiodic():
    N = 8
    rng = np.random.default_rng(500)
    c = I.draw_coeffs(N, rng)
    c[I.packed_two_l(N) % 2 == 0] = 0
    f = T.inverse_separable(c, N, full=True)
    assert np.max(np.abs(f[:, :, N:] + f[:, :, :N])) < 1e-12 * np.max(np.abs(f))


def test_adjoint_identity_full():
    N = 8
    rng = np.random.default_rng(600)
    f = _rand_grid(N, rng)
    g = I.draw_coeffs(N, rng)
    lhs = np.vdot(T.forward_separable(f, full=True), g)
    rhs = np.vdot(f, T.adjoint_separable(g, N, full=True))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_plancherel_full():
    """pref sum_k w_k |f|^2 = sum_l (2l+1) |c|^2 for band-limited mixed f."""
    N = 8
    rng = np.random.default_rng(700)
    c = I.draw_coeffs(N, rng)
    f = T.inverse_separable(c, N, full=True)
    from oracle import quadrature as Q
    w = Q.weights(N, "cc")
    lhs = np.sum(w[None, :, None] * np.abs(f) ** 2) / (4 * N * N)
    rhs = np.sum((I.packed_two_l(N) + 1) * np.abs(c) ** 2)
    assert abs(lhs - rhs) < 1e-12 * rhs
