"""The ragged batch in one persistent launch (SU2_FLAG_PERSISTENT): every
coefficient of every function against the FP64 oracle.

Bandwidths {8, 16, 32, 64, 128} with group sizes that leave partial function
blocks (5, 7, 33, 70, 67 functions; tensor-core blocks hold 64, FP32 blocks 32
or 64), interleaved in a seeded random order.  Per bandwidth two base grids
(white noise) are analysed by the oracle in FP64; function j of a group holds
base[j % 2] times alpha_j = 2^e i^r (exact in complex64), so its exact answer
is alpha_j times the oracle's and a kernel that mixed up functions, planes or
blocks would fail.  Both contraction paths (tensor cores at N = 64, 128 with
FP32 below; FP32 everywhere), tolerance 1e-5 relative max-norm per function.
Also: repeated calls and a workspace filled with 0xFF give identical results,
CUDA-graph replay equals direct launches, and plans that do not qualify are
refused.
"""
import numpy as np
import pytest

import su2inputs as I
from oracle import pool as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
COUNTS = {8: 5, 16: 7, 32: 33, 64: 70, 128: 67}


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def alpha(j):
    h = j // 2
    return (2.0 ** (h % 8 - 4)) * (1j ** ((h // 8) % 4))


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(71)
    Ns = np.concatenate([np.full(c, n) for n, c in COUNTS.items()])
    Ns = Ns[rng.permutation(len(Ns))]
    bases, refs = {}, {}
    for n in COUNTS:
        b = np.stack([I.draw_grid_gaussian((n, n, n), rng) for _ in range(2)]).astype(np.complex64)
        bases[n] = b
        refs[n] = OP.forward_all(b.astype(np.complex128))           # [2, C(n)]
    return [int(n) for n in Ns], bases, refs


def fill(plan, Ns, bases):
    x = torch.empty(plan.grid_elems, dtype=torch.complex64, device="cuda")
    slot = {n: 0 for n in COUNTS}
    order = []
    for f, n in enumerate(Ns):
        j = slot[n]
        slot[n] += 1
        g = (bases[n][j % 2] * np.complex64(alpha(j))).reshape(-1)
        o = plan.grid_offsets[f]
        x[o:o + n ** 3].copy_(torch.from_numpy(g))
        order.append(j)
    return x, order


def check_all(plan, out, Ns, order, refs):
    got = out.cpu().numpy()
    worst = 0.0
    for f, n in enumerate(Ns):
        j = order[f]
        o = plan.coeff_offsets[f]
        ref = refs[n][j % 2] * alpha(j)
        c = got[o:o + I.num_coeffs(n)].astype(np.complex128)
        rel = float(np.max(np.abs(c - ref)) / np.max(np.abs(ref)))
        worst = max(worst, rel)
        assert rel < TOL, (f, n, j, rel)
    return worst


@pytest.mark.parametrize("algo", ["tc_bf16x3", "fp32"])
def test_persistent_every_coefficient(su2, case, algo):
    Ns, bases, refs = case
    plan = su2.Plan(Ns=Ns, dtype="c64", algo=algo, persistent=True)
    assert plan.persistent
    x, order = fill(plan, Ns, bases)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    out1 = plan.forward(x, ws=ws).clone()
    out2 = plan.forward(x, ws=ws).clone()            # counters are re-zeroed per launch
    ws.fill_(0xFF)
    out3 = plan.forward(x, ws=ws).clone()
    plan.sync_status()
    assert torch.equal(out1, out2)
    assert torch.equal(out1, out3)
    check_all(plan, out1, Ns, order, refs)
    # the per-group launches of the same plan layout agree within the tolerance
    plain = su2.Plan(Ns=Ns, dtype="c64", algo=algo)
    assert not plain.persistent
    assert plain.grid_offsets == plan.grid_offsets and plain.coeff_offsets == plan.coeff_offsets
    ref = plain.forward(x)
    plain.sync_status()
    d = (out1 - ref).abs().max().item() / ref.abs().max().item()
    assert d < TOL, d
    plan.close()
    plain.close()


def test_persistent_graph_replay(su2, case):
    Ns, bases, refs = case
    plan = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3", persistent=True, graph=True)
    direct = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3", persistent=True)
    x, order = fill(plan, Ns, bases)
    a = plan.forward(x).clone()
    b = plan.forward(x).clone()                       # replay
    c = direct.forward(x)
    plan.sync_status()
    direct.sync_status()
    assert torch.equal(a, b)
    assert torch.equal(a, c)
    plan.close()
    direct.close()


@pytest.mark.parametrize("Ns", [[8], [128] * 3, [64] * 65, [16, 8, 32, 16]])
def test_persistent_small_plans(su2, Ns):
    """Single groups, one function, a block of 64 plus one, all-FP32 mixes."""
    rng = np.random.default_rng(len(Ns) * 7 + Ns[0])
    plan = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3", persistent=True)
    x = torch.empty(plan.grid_elems, dtype=torch.complex64, device="cuda")
    grids = []
    for f, n in enumerate(Ns):
        g = I.draw_grid_gaussian((n, n, n), rng).astype(np.complex64)
        grids.append(g)
        x[plan.grid_offsets[f]:plan.grid_offsets[f] + n ** 3].copy_(torch.from_numpy(g.reshape(-1)))
    got = plan.forward(x).cpu().numpy()
    plan.sync_status()
    check = sorted({0, len(Ns) - 1, len(Ns) // 2})
    for f in check:
        n = Ns[f]
        ref = OP.forward_all(grids[f][None].astype(np.complex128))[0]
        o = plan.coeff_offsets[f]
        c = got[o:o + I.num_coeffs(n)].astype(np.complex128)
        rel = float(np.max(np.abs(c - ref)) / np.max(np.abs(ref)))
        assert rel < TOL, (f, n, rel)
    plan.close()


def test_persistent_autotune_choice(su2, case):
    Ns, bases, refs = case
    plan = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3", autotune=True)
    assert plan.persistent in (True, False)
    x, order = fill(plan, Ns, bases)
    out = plan.forward(x)
    plan.sync_status()
    check_all(plan, out, Ns, order, refs)
    plan.close()


@pytest.mark.parametrize("kw", [dict(N=256, batch=1), dict(N=4, batch=2), dict(N=16, batch=1, dtype="c128", algo="fp64"),
                                dict(N=64, batch=1, literal=True), dict(N=64, batch=1, full_group=True)])
def test_persistent_refused_outside_its_range(su2, kw):
    kw = dict(kw)
    kw.setdefault("dtype", "c64")
    with pytest.raises(RuntimeError):
        su2.Plan(persistent=True, **kw)
