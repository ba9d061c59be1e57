"""Pins for the oracle's forward transform, synthesis and adjoint.

* direct O(N^6) sum == separated O(N^4) form on random (not band-limited)
  grids: the Sec. 4 factorisation is an exact identity;
* synthesis then analysis recovers coefficients of one sector exactly
  (Sec. 3 expansion and orthonormality; CC weights exact for the products);
* Plancherel per sector, the constant function, the cyclic-shift phase
  rule, linearity, the adjoint identity and a finite-difference gradient.
"""
import numpy as np
import pytest

import su2inputs as I
from oracle import grid, transform as T


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_direct_equals_separable(N):
    rng = np.random.default_rng(N)
    f = I.draw_grid_gaussian((N, N, N), rng)
    assert rel(T.forward_separable(f), T.forward_direct(f)) < 1e-13


@pytest.mark.parametrize("weights,literal", [("riemann", False), ("cc", True), ("riemann", True)])
def test_direct_equals_separable_other_grids(weights, literal):
    N = 8
    f = I.draw_grid_gaussian((N, N, N), np.random.default_rng(7))
    a = T.forward_direct(f, weights=weights, literal=literal)
    b = T.forward_separable(f, weights=weights, literal=literal)
    assert rel(b, a) < 1e-13


def test_inverse_separable_equals_direct():
    N = 8
    c = I.draw_coeffs(N, np.random.default_rng(3))
    assert rel(T.inverse_separable(c, N), T.inverse_direct(c, N)) < 1e-12


@pytest.mark.parametrize("N", [8, 16, 32])
@pytest.mark.parametrize("parity", [0, 1])
def test_roundtrip_per_sector(N, parity):
    rng = np.random.default_rng(100 + N + parity)
    c = I.draw_coeffs(N, rng)
    two_l = I.packed_two_l(N)
    cs = np.where(two_l % 2 == parity, c, 0)
    back = T.forward_separable(T.inverse_separable(cs, N))
    sel = two_l % 2 == parity
    assert np.max(np.abs(back[sel] - cs[sel])) < 1e-12 * np.max(np.abs(cs))
    # the other sector receives leakage on the paper's half-group domain
    assert np.max(np.abs(back[~sel])) > 1e-3


@pytest.mark.parametrize("parity", [0, 1])
def test_plancherel_per_sector(parity):
    N = 16
    rng = np.random.default_rng(5 + parity)
    c = I.draw_coeffs(N, rng)
    two_l = I.packed_two_l(N)
    cs = np.where(two_l % 2 == parity, c, 0)
    f = T.inverse_separable(cs, N)
    from oracle import quadrature
    w = quadrature.clenshaw_curtis(N)
    lhs = np.sum(w[None, :, None] * np.abs(f) ** 2) / (2 * N * N)
    rhs = np.sum((two_l + 1) * np.abs(cs) ** 2)
    assert abs(lhs - rhs) < 1e-12 * rhs


def test_constant_function():
    N = 16
    f = np.ones((N, N, N), dtype=np.complex128)
    r = T.forward_separable(f)
    two_l = I.packed_two_l(N)
    assert abs(r[0] - 1.0) < 1e-14
    assert np.max(np.abs(r[1:][two_l[1:] % 2 == 0])) < 1e-14
    assert np.max(np.abs(r[two_l % 2 == 1])) > 1e-2          # half-sector leakage


def test_cyclic_shift_phase_integer_sector():
    N = 16
    f = I.draw_grid_gaussian((N, N, N), np.random.default_rng(9))
    s1, s2 = 3, 5
    g = np.roll(np.roll(f, s1, axis=0), s2, axis=2)           # g[j1] = f[j1 - s1]
    rf, rg = T.forward_separable(f), T.forward_separable(g)
    for j in range(0, N, 2):
        for m2 in grid.half_range(j):
            for n2 in grid.half_range(j):
                i = grid.coeff_index(j, m2, n2)
                ph = np.exp(1j * 2 * np.pi * (n2 // 2 * s1 + m2 // 2 * s2) / N)
                assert abs(rg[i] - ph * rf[i]) < 1e-13


def test_linearity():
    N = 8
    rng = np.random.default_rng(11)
    f, g = I.draw_grid_gaussian((N, N, N), rng), I.draw_grid_gaussian((N, N, N), rng)
    a, b = 0.3 - 1.2j, 2.1 + 0.4j
    lhs = T.forward_separable(a * f + b * g)
    rhs = a * T.forward_separable(f) + b * T.forward_separable(g)
    assert rel(lhs, rhs) < 1e-14


@pytest.mark.parametrize("N", [8, 16])
def test_adjoint_identity(N):
    rng = np.random.default_rng(21 + N)
    f = I.draw_grid_gaussian((N, N, N), rng)
    g = I.draw_coeffs(N, rng)
    lhs = np.vdot(g, T.forward_separable(f))
    rhs = np.vdot(T.adjoint_separable(g, N), f)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_adjoint_equals_direct_transpose():
    # brute force: the forward matrix column by column at N = 4
    N = 4
    C = grid.num_coeffs(N)
    A = np.zeros((C, N ** 3), dtype=np.complex128)
    for p in range(N ** 3):
        e = np.zeros(N ** 3, dtype=np.complex128)
        e[p] = 1.0
        A[:, p] = T.forward_direct(e.reshape(N, N, N))
    g = I.draw_coeffs(N, np.random.default_rng(2))
    assert rel(T.adjoint_separable(g, N).reshape(-1), A.conj().T @ g) < 1e-13


def test_forward_pair_matches_full():
    N = 16
    f = I.draw_grid_gaussian((N, N, N), np.random.default_rng(31))
    full = T.forward_separable(f)
    for n2, m2 in [(0, 0), (3, -5), (-14, 2), (15, 15), (-1, 1)]:
        j0, vals = T.forward_pair(f, n2, m2)
        for i, v in enumerate(vals):
            assert abs(v - full[grid.coeff_index(j0 + 2 * i, m2, n2)]) < 1e-14


def test_finite_difference_gradient():
    N = 4
    rng = np.random.default_rng(41)
    f = I.draw_grid_gaussian((N, N, N), rng)
    tgt = I.draw_coeffs(N, rng)
    L0, g = T.loss_and_grad(f, tgt)
    h = 1e-6
    fd = np.zeros_like(g)
    flat = f.reshape(-1)
    for p in range(flat.size):
        for part, unit in ((0, 1.0), (1, 1j)):
            fp = flat.copy(); fp[p] += h * unit
            fm = flat.copy(); fm[p] -= h * unit
            Lp, _ = T.loss_and_grad(fp.reshape(f.shape), tgt)
            Lm, _ = T.loss_and_grad(fm.reshape(f.shape), tgt)
            d = (Lp - Lm) / (2 * h)
            fd.reshape(-1)[p] += d if part == 0 else 1j * d
    assert rel(fd, g) < 1e-7


def _doubled_n(N):
    return list(range(-(N - 1), N))


@pytest.mark.parametrize("N", [4, 8])
def test_forward_rows_equals_direct(N):
    """Stage 2 split over disjoint lists of n (what the host-pool runner does)
    reassembles the direct O(N^6) sum, for each grid of a batch."""
    rng = np.random.default_rng(70 + N)
    fs = np.stack([I.draw_grid_gaussian((N, N, N), rng) for _ in range(2)])
    ns = _doubled_n(N)
    out = np.zeros((2, grid.num_coeffs(N)), dtype=np.complex128)
    seen = np.zeros(grid.num_coeffs(N), dtype=np.int64)
    for part in (ns[0::3], ns[1::3], ns[2::3]):
        idx, vals = T.forward_rows(fs, part)
        out[:, idx] = vals
        seen[idx] += 1
    assert np.all(seen == 1)                      # every coefficient exactly once
    for b in range(2):
        assert rel(out[b], T.forward_direct(fs[b])) < 1e-13


def test_synthesis_rows_equal_direct_and_transpose():
    """Synthesis rows reassembled at a subset of beta nodes equal the direct
    synthesis sum there; adjoint rows equal the brute-force conjugate
    transpose of the direct forward matrix (N = 4)."""
    N = 4
    rng = np.random.default_rng(81)
    cs = np.stack([I.draw_coeffs(N, rng) for _ in range(2)])
    ks = [0, 2, 3]
    ns = _doubled_n(N)
    parts = [T.synthesis_rows(cs, N, part, ks, modes=("synthesis", "adjoint")) for part in (ns[:3], ns[3:])]
    syn = T.planes_from_rows([p["synthesis"] for p in parts], N)
    adj = T.planes_from_rows([p["adjoint"] for p in parts], N)
    C = grid.num_coeffs(N)
    A = np.zeros((C, N ** 3), dtype=np.complex128)
    for p in range(N ** 3):
        e = np.zeros(N ** 3, dtype=np.complex128)
        e[p] = 1.0
        A[:, p] = T.forward_direct(e.reshape(N, N, N))
    for b in range(2):
        assert rel(syn[b], T.inverse_direct(cs[b], N)[:, ks, :]) < 1e-12
        assert rel(adj[b], (A.conj().T @ cs[b]).reshape(N, N, N)[:, ks, :]) < 1e-13
