"""Forward transform on the full-group grid (psi over [-2 pi, 2 pi), 2N
nodes, prefactor 1/(4N^2)) against the oracle's same definition: full grids
of random data, sampled pairs at N = 128, 256, exact recovery of coefficients
mixing both sectors (which the paper's half domain cannot give), a ragged
batch, and the forward-only restriction.  Tolerance 1e-5 relative to the
largest oracle coefficient, as for the other complex64 tests."""
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


def _grid(N, rng):
    return I.draw_grid_gaussian((N, N, 2 * N), rng).astype(np.complex64).astype(np.complex128)


def _run(su2, grids, Ns, algo):
    plan = su2.Plan(Ns=Ns, dtype="c64", algo=algo, full_group=True)
    flat = np.zeros(plan.grid_elems, dtype=np.complex64)
    for g, o in zip(grids, plan.grid_offsets):
        flat[o:o + g.size] = g.reshape(-1)
    out = plan.forward(torch.from_numpy(flat).cuda())
    plan.sync_status()
    out = out.cpu().numpy().astype(np.complex128)
    return plan, [out[o:o + I.num_coeffs(n)] for o, n in zip(plan.coeff_offsets, Ns)]


@pytest.mark.parametrize("algo", ["fp32", "tc_bf16x3"])
def test_full_group_n64_vs_oracle(su2, algo):
    N = 64
    rng = np.random.default_rng(70)
    grids = [_grid(N, rng) for _ in range(2)]
    plan, outs = _run(su2, grids, [N, N], algo)
    assert plan.grid_elems == 2 * 2 * N ** 3
    for g, o in zip(grids, outs):
        assert _rel(o, T.forward_separable(g, full=True)) < TOL


@pytest.mark.parametrize("N,algo", [(128, "fp32"), (256, "tc_bf16x3")])
def test_full_group_sampled(su2, N, algo):
    rng = np.random.default_rng(71 + N)
    g = _grid(N, rng)
    _, (o,) = _run(su2, [g], [N], algo)
    worst = scale = 0.0
    for n2, m2 in [(0, 0), (N - 2, N - 2), (-(N - 1), N - 1), (N - 1, -(N - 1)), (1, 1), (-7, 13), (30, -2)]:
        j0, vals = T.forward_pair(g, n2, m2, full=True)
        for i, v in enumerate(vals):
            worst = max(worst, abs(o[OG.coeff_index(j0 + 2 * i, m2, n2)] - v))
            scale = max(scale, abs(v))
    assert worst / scale < TOL


def test_full_group_recovers_mixed_sectors(su2):
    """Band-limited coefficients in both sectors at once: the full-group
    forward of their synthesis gives them back (on the paper's domain the
    sectors leak into each other)."""
    N = 64
    rng = np.random.default_rng(72)
    c = I.draw_coeffs(N, rng)
    g = T.inverse_separable(c, N, full=True)
    _, (o,) = _run(su2, [g.astype(np.complex64).astype(np.complex128)], [N], "tc_bf16x3")
    assert _rel(o, c) < TOL


@pytest.mark.parametrize("algo", ["fp32", "tc_bf16x3"])
def test_full_group_inverse_and_adjoint_n128(su2, algo):
    """Synthesis and adjoint on the full-group grid against the oracle, every
    grid point of two functions (2N = 256 psi nodes)."""
    N, B = 128, 2
    rng = np.random.default_rng(74)
    cs = [I.draw_coeffs(N, rng, "inv1").astype(np.complex64) for _ in range(B)]
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo=algo, full_group=True)
    c_dev = torch.from_numpy(np.concatenate(cs)).cuda()
    syn = plan.inverse(c_dev).cpu().numpy().astype(np.complex128)
    adj = plan.backward(c_dev).cpu().numpy().astype(np.complex128)
    plan.sync_status()
    for b in range(B):
        o = plan.grid_offsets[b]
        c64 = cs[b].astype(np.complex128)
        got_s = syn[o:o + 2 * N ** 3].reshape(N, N, 2 * N)
        got_a = adj[o:o + 2 * N ** 3].reshape(N, N, 2 * N)
        assert _rel(got_s, T.inverse_separable(c64, N, full=True)) < TOL, ("synthesis", b)
        assert _rel(got_a, T.adjoint_separable(c64, N, full=True)) < TOL, ("adjoint", b)


@pytest.mark.parametrize("N", [128, 256])
def test_full_group_round_trip_mixed_sectors(su2, N):
    """forward(inverse(c)) = c for coefficients in both sectors at once: exact
    on the full group (Peter-Weyl orthogonality over all of SU(2))."""
    rng = np.random.default_rng(75 + N)
    c = I.draw_coeffs(N, rng, "inv1").astype(np.complex64)
    plan = su2.Plan(N=N, batch=1, dtype="c64", algo="fp32", full_group=True)
    back = plan.forward(plan.inverse(torch.from_numpy(c).cuda()))
    plan.sync_status()
    back = back.cpu().numpy()
    assert np.max(np.abs(back - c)) / np.max(np.abs(c)) < TOL


def test_full_group_ragged_and_inverse_limits(su2):
    Ns = [64, 128, 64]
    rng = np.random.default_rng(73)
    grids = [_grid(n, rng) for n in Ns]
    plan, outs = _run(su2, grids, Ns, "fp32")
    for n, g, o in zip(Ns, grids, outs):
        if n == 64:
            assert _rel(o, T.forward_separable(g, full=True)) < TOL
        else:
            j0, vals = T.forward_pair(g, 3, -5, full=True)
            got = np.array([o[OG.coeff_index(j0 + 2 * i, -5, 3)] for i in range(len(vals))])
            assert _rel(got, vals) < TOL
    with pytest.raises(su2.SU2Error):                 # synthesis on the full group: N = 128, 256
        plan.inverse(torch.zeros(plan.coeff_elems, dtype=torch.complex64, device="cuda"))
