"""FP32 beta contraction of large batches (48 functions or more), which runs one
launch per row class of tiles: tiles with at most 32 rows of l take 64 functions
per block, 32 < L <= 64 take 32, longer tiles 16.

The per-coefficient arithmetic (recurrence steps, order of the node sum) is the
same as in the kernel of small batches, so every function of a 64-function
plan must equal, bit for bit, the same grid transformed by a 4-function plan;
one function of each size is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import su2inputs as I
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("N", [128, 256])
def test_row_classes_match_small_batch_kernel(su2, N):
    B, NB = 64, 4
    rng = np.random.default_rng(40 + N)
    base = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(NB)]
    small = su2.Plan(N=N, batch=NB, dtype="c64", algo="fp32")
    xs = torch.from_numpy(np.concatenate([g.reshape(-1) for g in base])).cuda()
    ref = small.forward(xs)
    small.sync_status()
    big = su2.Plan(N=N, batch=B, dtype="c64", algo="fp32")
    x = torch.empty(B * N ** 3, dtype=torch.complex64, device="cuda")
    for b in range(B):
        x[b * N ** 3:(b + 1) * N ** 3].copy_(xs[(b % NB) * N ** 3:(b % NB + 1) * N ** 3])
    out = big.forward(x)
    big.sync_status()
    C = I.num_coeffs(N)
    for b in range(B):
        assert torch.equal(out[b * C:(b + 1) * C], ref[(b % NB) * C:(b % NB + 1) * C]), b
    if N == 128:          # the whole coefficient vector of one function against the oracle
        want = T.forward_separable(base[1].astype(np.complex128))
        got = out[C:2 * C].cpu().numpy()
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < TOL32
