"""Ragged batches: 512 functions with N drawn from {16, 32, 64, 128}, complex64,
through a plan that records its forward transform in a CUDA graph and tunes
its kernels, against the oracle on sampled functions of every bandwidth and
against the plain plan on all of them."""
import numpy as np
import pytest

import su2inputs as I
from oracle import grid as OG
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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_ragged_512_graph_autotune(su2):
    rng = np.random.default_rng(3)
    Ns = I.draw_ragged_bandwidths(512, (16, 32, 64, 128), rng)
    plan = su2.Plan(Ns=Ns, dtype="c64", graph=True, autotune=True)
    plain = su2.Plan(Ns=Ns, dtype="c64")
    assert plan.grid_offsets == plain.grid_offsets
    x = torch.empty(plan.grid_elems, dtype=torch.complex64, device="cuda")
    grids = {}
    sample = {}
    for n in (16, 32, 64, 128):
        fs = [f for f, m in enumerate(Ns) if m == n]
        sample[n] = fs[:3] + fs[-1:]
    for f, n in enumerate(Ns):
        g = I.draw_grid_gaussian((n, n, n), rng).astype(np.complex64)
        o = plan.grid_offsets[f]
        x[o:o + n ** 3].copy_(torch.from_numpy(g.reshape(-1)))
        if f in sample[n]:
            grids[f] = g.astype(np.complex128)
    out1 = plan.forward(x)
    out2 = plan.forward(x)                     # replay of the recorded graph
    ref = plain.forward(x)
    plan.sync_status()
    plain.sync_status()
    assert torch.equal(out1, out2)
    d = (out1 - ref).abs().max().item() / ref.abs().max().item()
    assert d < TOL, d
    got = out1.cpu().numpy()
    for n in (16, 32, 64, 128):
        for f in sample[n]:
            o = plan.coeff_offsets[f]
            c = got[o:o + I.num_coeffs(n)].astype(np.complex128)
            if n <= 64:
                assert _rel(c, T.forward_separable(grids[f])) < TOL, (n, f)
            else:
                worst = scale = 0.0
                for n2, m2 in [(0, 0), (126, -126), (127, 127), (-5, 3), (44, 44), (-1, -127)]:
                    j0, vals = T.forward_pair(grids[f], n2, m2)
                    for i, v in enumerate(vals):
                        worst = max(worst, abs(c[OG.coeff_index(j0 + 2 * i, m2, n2)] - v))
                        scale = max(scale, abs(v))
                assert worst / scale < TOL, (n, f)


@pytest.mark.parametrize("algo", ["fp32", "tc_bf16x3"])
def test_graph_replay_follows_new_inputs(su2, algo):
    """A recorded graph reads the buffers it was recorded with: new contents in
    the same buffers give the new transform; new buffers record a new graph."""
    N, B = 64, 3
    rng = np.random.default_rng(60)
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo=algo, graph=True)
    plain = su2.Plan(N=N, batch=B, dtype="c64", algo=algo)
    x = torch.empty(plan.grid_elems, dtype=torch.complex64, device="cuda")
    out = torch.empty(plan.coeff_elems, dtype=torch.complex64, device="cuda")
    for rep in range(3):
        x.copy_(torch.from_numpy(np.concatenate(
            [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64).reshape(-1) for _ in range(B)])))
        plan.forward(x, out=out)
        ref = plain.forward(x)
        plan.sync_status()
        assert torch.equal(out, ref), rep
    x2 = x.clone()
    out2 = plan.forward(x2)
    plan.sync_status()
    assert torch.equal(out2, plain.forward(x2))


def test_ragged_tensor_core_autotune_and_cache(su2, tmp_path, monkeypatch):
    """A tensor-core plan over the ragged batch with the autotuner (which may move
    a group to the FP32 contraction) against the oracle-checked plain plan; the
    choices (per group, and one-launch or per-group launches for the whole
    plan) go to the SU2_TUNE_CACHE file, and a second plan that reads them
    gives the same coefficients bit for bit."""
    import json
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SU2_TUNE_CACHE", str(cache))
    rng = np.random.default_rng(31)
    Ns = I.draw_ragged_bandwidths(96, (16, 32, 64, 128), rng)
    plan = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3", graph=True, autotune=True)
    plain = su2.Plan(Ns=Ns, dtype="c64", algo="fp32")
    x = torch.randn(plan.grid_elems, dtype=torch.complex64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(31))
    out = plan.forward(x)
    ref = plain.forward(x)
    plan.sync_status()
    d = (out - ref).abs().max().item() / ref.abs().max().item()
    assert d < TOL, d
    entries = json.loads(cache.read_text())
    # one per bandwidth group, and the whole plan's persistent-launch choice
    assert len(entries) == 5
    assert sum("|ragged|" in k for k in entries) == 1
    for v in entries.values():
        assert set(v) == {"tc", "s1", "rc", "bt"}
    again = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3", autotune=True)
    assert again.persistent == plan.persistent
    out2 = again.forward(x)
    again.sync_status()
    assert torch.equal(out2, out)
    assert json.loads(cache.read_text()) == entries
