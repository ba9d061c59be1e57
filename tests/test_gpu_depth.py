"""Stage 2 by the depth-k divide-and-conquer projection (su2_forward_stage2_depth)
against the oracle's plain definition and the library's depth-1 recurrence
contraction, on complex128 plans (FP64; tolerance 1e-12 relative to the
largest oracle coefficient, as for the other FP64 tests): whole transforms at
N = 4..64 for k = 1..5, a ragged batch with more functions than one CTA takes,
sampled pairs at N = 256, and the argument checks."""
import numpy as np
import pytest

import su2inputs as I
from oracle import grid as OG
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _stage1(su2, grids, Ns):
    plan = su2.Plan(Ns=Ns, dtype="c128", algo="fp64")
    flat = np.zeros(plan.grid_elems, dtype=np.complex128)
    for g, o in zip(grids, plan.grid_offsets):
        flat[o:o + g.size] = g.reshape(-1)
    ws = plan.forward_stage1(torch.from_numpy(flat).cuda())
    return plan, ws


def _split(plan, out, Ns):
    out = out.cpu().numpy()
    return [out[o:o + I.num_coeffs(n)] for o, n in zip(plan.coeff_offsets, Ns)]


@pytest.mark.parametrize("N", [4, 16, 64])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_depth_vs_oracle(su2, N, k):
    rng = np.random.default_rng(500 + N + k)
    B = 6
    grids = [I.draw_grid_gaussian((N, N, N), rng) for _ in range(B)]
    plan, ws = _stage1(su2, grids, [N] * B)
    ref = plan.forward_stage2(ws=ws)
    got = plan.forward_stage2_depth(k, ws=ws)
    plan.sync_status()
    for g, o, r in zip(grids, _split(plan, got, [N] * B), _split(plan, ref, [N] * B)):
        want = T.forward_separable(g)
        assert _rel(o, want) < TOL
        assert _rel(o, r) < TOL


def test_depth_ragged(su2):
    Ns = [32, 8, 32, 32, 16, 32, 32, 8, 32]          # 6 functions at N = 32: two CTAs' worth
    rng = np.random.default_rng(510)
    grids = [I.draw_grid_gaussian((n, n, n), rng) for n in Ns]
    plan, ws = _stage1(su2, grids, Ns)
    for k in (2, 3):
        got = _split(plan, plan.forward_stage2_depth(k, ws=ws), Ns)
        plan.sync_status()
        for g, o in zip(grids, got):
            assert _rel(o, T.forward_separable(g)) < TOL


@pytest.mark.parametrize("k", [1, 3])
def test_depth_n256_sampled(su2, k):
    N = 256
    rng = np.random.default_rng(520 + k)
    g = I.draw_grid_gaussian((N, N, N), rng)
    plan, ws = _stage1(su2, [g], [N])
    o = plan.forward_stage2_depth(k, ws=ws).cpu().numpy()
    plan.sync_status()
    worst = scale = 0.0
    for n2, m2 in [(0, 0), (254, 254), (-255, 255), (255, -255), (1, 1), (-37, 63), (50, -2), (-99, -99), (200, 10)]:
        j0, vals = T.forward_pair(g, n2, m2)
        for i, v in enumerate(vals):
            worst = max(worst, abs(o[OG.coeff_index(j0 + 2 * i, m2, n2)] - v))
            scale = max(scale, abs(v))
    assert worst / scale < TOL


def test_depth_argument_checks(su2):
    plan = su2.Plan(N=16, batch=1, dtype="c128", algo="fp64")
    ws = plan.workspace()
    for bad in (0, 6):
        with pytest.raises(su2.SU2Error):
            plan.forward_stage2_depth(bad, ws=ws)
    p64 = su2.Plan(N=16, batch=1, dtype="c64", algo="fp32")
    with pytest.raises(su2.SU2Error):
        p64.forward_stage2_depth(2)
