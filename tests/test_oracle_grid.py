"""Pins for the sampling grid and packed layout (oracle.grid).

Sec. 4 sampling grid: phi and psi start at -pi; theta_k = k pi/(N-1) runs from
0 to pi.  Periodic spacing 2 pi/N by default, printed spacing 2 pi/(N-1) with
literal=True (last node on +pi).
"""
import numpy as np

from oracle import grid


def test_nodes():
    assert np.allclose(grid.alpha_nodes(4), [-np.pi, -np.pi / 2, 0.0, np.pi / 2])
    assert np.allclose(grid.gamma_nodes(4), [-np.pi, -np.pi / 2, 0.0, np.pi / 2])
    assert np.allclose(grid.alpha_nodes(4, literal=True), [-np.pi, -np.pi / 3, np.pi / 3, np.pi])
    b = grid.beta_nodes(5)
    assert np.allclose(b, [0, np.pi / 4, np.pi / 2, 3 * np.pi / 4, np.pi])


def test_packed_layout():
    N = 6
    assert grid.num_coeffs(N) == sum((j + 1) ** 2 for j in range(N))
    seen = set()
    for j in range(N):
        for a in grid.half_range(j):
            for b in grid.half_range(j):
                seen.add(grid.coeff_index(j, a, b))
    assert seen == set(range(grid.num_coeffs(N)))
    # row m + l, column n + l inside block j = 2l
    assert grid.coeff_index(2, -2, 2) == 5 + 2
    assert grid.coeff_index(2, 2, -2) == 5 + 6
