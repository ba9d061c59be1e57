"""The host-pool runner of the oracle (oracle.pool) reassembles the same
values as the single-process separated forms, which are themselves pinned to
the direct sums (test_oracle_transform.py)."""
import numpy as np

import su2inputs as I
from oracle import grid, pool, transform as T


def test_forward_all_and_sample_match_separable():
    N = 16
    rng = np.random.default_rng(90)
    fs = np.stack([I.draw_grid_gaussian((N, N, N), rng) for _ in range(2)])
    out = pool.forward_all(fs, workers=2)
    part = pool.forward_all(fs, workers=2, row_stride=4)
    for b in range(2):
        ref = T.forward_separable(fs[b])
        assert np.max(np.abs(out[b] - ref)) < 1e-13 * np.max(np.abs(ref))
        hit = part[b] != 0
        assert 0.15 < hit.mean() < 0.4
        assert np.max(np.abs(part[b][hit] - ref[hit])) < 1e-13 * np.max(np.abs(ref))


def test_synthesis_planes_match_separable():
    N = 16
    rng = np.random.default_rng(91)
    cs = np.stack([I.draw_coeffs(N, rng) for _ in range(2)])
    ks = [0, 7, 15]
    got = pool.synthesis_planes(cs, N, ks, modes=("synthesis", "adjoint"), workers=2)
    for b in range(2):
        syn = T.inverse_separable(cs[b], N)[:, ks, :]
        adj = T.adjoint_separable(cs[b], N)[:, ks, :]
        assert np.max(np.abs(got["synthesis"][b] - syn)) < 1e-12 * np.max(np.abs(syn))
        assert np.max(np.abs(got["adjoint"][b] - adj)) < 1e-13 * np.max(np.abs(adj))
    assert grid.num_coeffs(N) == cs.shape[1]
