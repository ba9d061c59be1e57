"""Stage 1 alone (su2_forward_stage1) against the oracle's torus double sum.

The planes F2_s[k][m][n] = w_k/(2N^2) sum f e^{i(n alpha + m gamma)} are
compared element by element on sampled beta nodes (both sectors, every (m, n);
the unused Nyquist row and column of sector 0 must be zero), at the bandwidths
that run the two-phase complex64 kernel (N = 128, 256, 512) and on a ragged
batch whose bandwidth groups are not regularly strided in the grid buffer.
"""
import numpy as np
import pytest

import su2inputs as I
from oracle import grid as OG
from oracle import quadrature as OQ
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def expected_planes(f, k):
    """Both sectors of plane k in the workspace layout [mi][ni], from the oracle."""
    N = f.shape[0]
    al, ga = OG.alpha_nodes(N), OG.gamma_nodes(N)
    w = OQ.weights(N, "cc")
    out = []
    for sector in ("int", "half"):
        idx = T.sector_indices(N, sector)
        F = T.torus_dft(f[:, k:k + 1, :], idx, idx, al, ga)[0]          # [n, m]
        plane = np.zeros((N, N), dtype=np.complex128)
        pos = (idx + (0 if sector == "int" else -1)) // 2 + N // 2        # mi / ni of doubled index
        plane[np.ix_(pos, pos)] = (F.T) * w[k] / (2.0 * N * N)            # rows m, columns n
        out.append(plane)
    return out


def read_plane(c, base, N, k, s, tile_major):
    if not tile_major:
        o = base + (2 * k + s) * N * N
        return c[o:o + N * N].cpu().numpy().astype(np.complex128).reshape(N, N)
    # [s][mi][ni/4][k][ni%4]
    blk = c[base + s * N ** 3: base + (s + 1) * N ** 3].reshape(N, N // 4, N, 4)
    return blk[:, :, k, :].reshape(N, N).cpu().numpy().astype(np.complex128)


def check_planes(plan, ws, f, fi, ks, tile_major=False):
    N = f.shape[0]
    c = ws.view(torch.complex64)
    base = plan.plane_offsets[fi]
    worst = scale = 0.0
    for k in ks:
        for s, ref in enumerate(expected_planes(f, k)):
            got = read_plane(c, base, N, k, s, tile_major)
            worst = max(worst, float(np.max(np.abs(got - ref))))
            scale = max(scale, float(np.max(np.abs(ref))))
            if s == 0:
                assert np.all(got[0, :] == 0) and np.all(got[:, 0] == 0)
    assert worst / scale < TOL, (fi, worst / scale)


@pytest.mark.parametrize("N,B", [(64, 2), (128, 3), (256, 2), (512, 1)])
def test_stage1_planes_uniform(su2, N, B):
    rng = np.random.default_rng(40 + N)
    grids = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(B)]
    plan = su2.Plan(N=N, batch=B, dtype="c64")
    x = torch.from_numpy(np.concatenate([g.reshape(-1) for g in grids])).cuda()
    ws = plan.forward_stage1(x)
    plan.sync_status()
    ks = [0, 1, N // 2 - 1, N // 2, N - 2, N - 1] + list(rng.integers(0, N, 3))
    for fi, g in enumerate(grids):
        check_planes(plan, ws, g.astype(np.complex128), fi, ks)


def test_stage1_planes_ragged(su2):
    Ns = [128, 64, 128, 256, 128]
    rng = np.random.default_rng(47)
    grids = [I.draw_grid_gaussian((n, n, n), rng).astype(np.complex64) for n in Ns]
    plan = su2.Plan(Ns=Ns, dtype="c64")
    flat = np.zeros(plan.grid_elems, dtype=np.complex64)
    for g, o in zip(grids, plan.grid_offsets):          # grids are grouped by bandwidth
        flat[o:o + g.size] = g.reshape(-1)
    x = torch.from_numpy(flat).cuda()
    ws = plan.forward_stage1(x)
    plan.sync_status()
    for fi, (n, g) in enumerate(zip(Ns, grids)):
        check_planes(plan, ws, g.astype(np.complex128), fi, [0, 5, n // 2, n - 1])


def test_stage1_repeat_reuses_scratch(su2):
    """Back-to-back launches on one workspace (the counters are reset per launch)."""
    N, B = 256, 2
    rng = np.random.default_rng(48)
    plan = su2.Plan(N=N, batch=B, dtype="c64")
    for rep in range(3):
        grids = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(B)]
        x = torch.from_numpy(np.concatenate([g.reshape(-1) for g in grids])).cuda()
        ws = plan.forward_stage1(x)
        plan.sync_status()
        for fi, g in enumerate(grids):
            check_planes(plan, ws, g.astype(np.complex128), fi, [3, N - 4])


def test_stage1_workspace_only_16_byte_aligned(su2):
    """A workspace that is 16-byte but not 128-byte aligned (allowed by the C ABI):
    the intermediate ring then shares L2 lines with its neighbours and must not be
    discarded; the planes stay exact."""
    N, B = 256, 2
    rng = np.random.default_rng(49)
    grids = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(B)]
    plan = su2.Plan(N=N, batch=B, dtype="c64")
    raw = torch.empty(plan.workspace_bytes + 256, dtype=torch.uint8, device="cuda")
    ws = raw[16:16 + plan.workspace_bytes]
    assert ws.data_ptr() % 128 == 16
    x = torch.from_numpy(np.concatenate([g.reshape(-1) for g in grids])).cuda()
    plan.forward_stage1(x, ws=ws)
    plan.sync_status()
    for fi, g in enumerate(grids):
        check_planes(plan, ws, g.astype(np.complex128), fi, [0, 7, N // 2, N - 1])


@pytest.mark.parametrize("N,B", [(64, 3), (256, 2)])
def test_stage1_planes_tensor_core_layout(su2, N, B):
    """Plans of the tensor-core path keep the planes tile-major."""
    rng = np.random.default_rng(50 + N)
    grids = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(B)]
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo="tc_bf16x3")
    x = torch.from_numpy(np.concatenate([g.reshape(-1) for g in grids])).cuda()
    ws = plan.forward_stage1(x)
    plan.sync_status()
    for fi, g in enumerate(grids):
        check_planes(plan, ws, g.astype(np.complex128), fi, [0, 1, N // 2, N - 1], tile_major=True)


def test_stage1_two_phase_with_few_resident_blocks(su2):
    """The two-phase DFT hands out items in order, so it completes with any
    number of resident thread blocks; the grid is capped at 1 and 5 blocks (in a
    child process, the cap being read from the environment at launch)."""
    import os
    import subprocess
    import sys
    code = r'''
import numpy as np, torch, sys
sys.path.insert(0, ".")
import su2inputs as I
import paper_2605_23923_gb300 as su2
from tests.test_gpu_stage1 import check_planes
N, B = 128, 2
rng = np.random.default_rng(51)
grids = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(B)]
plan = su2.Plan(N=N, batch=B, dtype="c64")
x = torch.from_numpy(np.concatenate([g.reshape(-1) for g in grids])).cuda()
ws = plan.forward_stage1(x)
plan.sync_status()
for fi, g in enumerate(grids):
    check_planes(plan, ws, g.astype(np.complex128), fi, [0, 9, N // 2, N - 1])
print("ok")
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for cap in ("1", "5"):
        env = dict(os.environ, SU2_STAGE1_MAX_CTAS=cap)
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (cap, r.stdout[-2000:], r.stderr[-2000:])
