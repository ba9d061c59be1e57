"""Forward transform on the grid as Sec. 4 prints it (alpha, gamma spacing
2 pi/(N-1), the node +pi repeating -pi, prefactor 1/(2(N-1)^2)) against the
oracle's same sum: whole grids at N = 4..64 with both beta weightings and both
contraction paths, sampled pairs at N = 128 and 256, a ragged batch, grids
whose repeated nodes disagree (the fold must add them, not pick one); the
synthesis and the adjoint at every printed node (the repeated ones included)
at N = 64 and 128, and their restriction to N >= 64.  Tolerance 1e-5 relative
to the largest oracle value, as for the other complex64 tests."""
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
    return I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64).astype(np.complex128)


def _run(su2, grids, Ns, algo, weights="cc"):
    plan = su2.Plan(Ns=Ns, dtype="c64", algo=algo, weights=weights, literal=True)
    flat = np.zeros(plan.grid_elems, dtype=np.complex64)
    for g, o in zip(grids, plan.grid_offsets):
        flat[o:o + g.size] = g.reshape(-1)
    out = plan.forward(torch.from_numpy(flat).cuda())
    plan.sync_status()
    out = out.cpu().numpy().astype(np.complex128)
    return plan, [out[o:o + I.num_coeffs(n)] for o, n in zip(plan.coeff_offsets, Ns)]


@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("weights", ["cc", "riemann"])
def test_literal_small_vs_oracle(su2, N, weights):
    rng = np.random.default_rng(80 + N)
    grids = [_grid(N, rng) for _ in range(3)]
    _, outs = _run(su2, grids, [N] * 3, "fp32", weights)
    for g, o in zip(grids, outs):
        assert _rel(o, T.forward_separable(g, weights=weights, literal=True)) < TOL


@pytest.mark.parametrize("algo", ["fp32", "tc_bf16x3"])
def test_literal_n64_vs_oracle(su2, algo):
    N = 64
    rng = np.random.default_rng(90)
    grids = [_grid(N, rng) for _ in range(2)]
    _, outs = _run(su2, grids, [N, N], algo)
    for g, o in zip(grids, outs):
        assert _rel(o, T.forward_separable(g, literal=True)) < TOL


def test_literal_fold_uses_both_copies(su2):
    """The repeated nodes carry different values: the sum counts both of them
    (for half-integer n with opposite signs), so a kernel that dropped or
    overwrote either copy fails."""
    N = 16
    rng = np.random.default_rng(91)
    g = np.zeros((N, N, N), dtype=np.complex128)
    g[0] = _grid(N, rng)[0]
    g[N - 1] = 3.0 * _grid(N, rng)[0]
    g[:, :, 0] += _grid(N, rng)[:, :, 0]
    g[:, :, N - 1] -= 2.0 * _grid(N, rng)[:, :, 0]
    g = g.astype(np.complex64).astype(np.complex128)
    _, (o,) = _run(su2, [g], [N], "fp32")
    assert _rel(o, T.forward_separable(g, literal=True)) < TOL


@pytest.mark.parametrize("N,algo", [(128, "fp32"), (256, "tc_bf16x3")])
def test_literal_sampled(su2, N, algo):
    rng = np.random.default_rng(92 + N)
    g = _grid(N, rng)
    _, (o,) = _run(su2, [g], [N], algo)
    worst = scale = 0.0
    for n2, m2 in [(0, 0), (N - 2, N - 2), (-(N - 1), N - 1), (N - 1, -(N - 1)), (1, 1), (-7, 13), (30, -2)]:
        j0, vals = T.forward_pair(g, n2, m2, literal=True)
        for i, v in enumerate(vals):
            worst = max(worst, abs(o[OG.coeff_index(j0 + 2 * i, m2, n2)] - v))
            scale = max(scale, abs(v))
    assert worst / scale < TOL


@pytest.mark.parametrize("N,algo", [(64, "fp32"), (64, "tc_bf16x3"), (128, "fp32")])
def test_literal_inverse_and_adjoint(su2, N, algo):
    """Synthesis (Sec. 3 expansion) and the adjoint of the printed-grid forward
    map at every node of the printed grid, two functions, against the oracle."""
    B = 2
    rng = np.random.default_rng(94 + N)
    cs = [I.draw_coeffs(N, rng, "inv1").astype(np.complex64) for _ in range(B)]
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo=algo, literal=True)
    c_dev = torch.from_numpy(np.concatenate(cs)).cuda()
    syn = plan.inverse(c_dev).cpu().numpy().astype(np.complex128)
    adj = plan.backward(c_dev).cpu().numpy().astype(np.complex128)
    plan.sync_status()
    for b in range(B):
        o = plan.grid_offsets[b]
        c64 = cs[b].astype(np.complex128)
        got_s = syn[o:o + N ** 3].reshape(N, N, N)
        got_a = adj[o:o + N ** 3].reshape(N, N, N)
        assert _rel(got_s, T.inverse_separable(c64, N, literal=True)) < TOL, ("synthesis", b)
        assert _rel(got_a, T.adjoint_separable(c64, N, literal=True)) < TOL, ("adjoint", b)


def test_literal_adjoint_identity_n256(su2):
    """<A f, g> = <f, A^H g> on the printed grid at N = 256 (any size)."""
    N = 256
    plan = su2.Plan(N=N, batch=1, dtype="c64", algo="tc_bf16x3", literal=True)
    gen = torch.Generator(device="cuda").manual_seed(95)
    f = torch.randn(plan.grid_elems, dtype=torch.complex64, device="cuda", generator=gen)
    g = torch.randn(plan.coeff_elems, dtype=torch.complex64, device="cuda", generator=gen)
    af = plan.forward(f)
    lhs = torch.vdot(af.to(torch.complex128), g.to(torch.complex128))
    rhs = torch.vdot(f.to(torch.complex128), plan.backward(g).to(torch.complex128))
    plan.sync_status()
    scale = (af.abs().double().norm() * g.abs().double().norm()).item()
    assert abs((lhs - rhs).item()) < TOL * scale


def test_literal_ragged_and_inverse_limits(su2):
    Ns = [16, 64, 32, 16]
    rng = np.random.default_rng(93)
    grids = [_grid(n, rng) for n in Ns]
    plan, outs = _run(su2, grids, Ns, "tc_bf16x3")
    for g, o in zip(grids, outs):
        assert _rel(o, T.forward_separable(g, literal=True)) < TOL
    with pytest.raises(su2.SU2Error):                 # synthesis on the printed grid: N >= 64
        plan.inverse(torch.zeros(plan.coeff_elems, dtype=torch.complex64, device="cuda"))
