"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are seeded (su2inputs) and, where band-limited, synthesised by the
oracle in FP64; the grid is cast to the GPU dtype first and the oracle
analyses the same cast values.  Error metric: max |gpu - oracle| over all
coefficients of a function divided by max |oracle| (then max over the batch).
Tolerances: 1e-12 for the FP64 path, 1e-5 for the FP32 path.
"""
import numpy as np
import pytest

import su2inputs as I
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def cast(x, dtype):
    return x.astype(np.complex64).astype(np.complex128) if dtype == "c64" else x.astype(np.complex128)


def to_dev(x, dtype):
    t = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64 if dtype == "c64" else np.complex128)))
    return t.reshape(-1).cuda()


def tol(dtype):
    return TOL64 if dtype == "c128" else TOL32


def run_forward(su2, grids, dtype, Ns=None, weights="cc", algo="auto"):
    if Ns is None:
        plan = su2.Plan(N=grids[0].shape[0], batch=len(grids), dtype=dtype, weights=weights, algo=algo)
    else:
        plan = su2.Plan(Ns=Ns, dtype=dtype, weights=weights, algo=algo)
    flat = np.zeros(plan.grid_elems, dtype=np.complex128)
    for g, o in zip(grids, plan.grid_offsets):          # the plan decides where each grid goes
        flat[o:o + g.size] = g.reshape(-1)
    out = plan.forward(to_dev(flat, dtype))
    plan.sync_status()
    out = out.cpu().numpy().astype(np.complex128)
    return plan, [out[o:o + I.num_coeffs(n)] for o, n in zip(plan.coeff_offsets, plan.Ns)]


# ---------------------------------------------------------------------------
# Forward
# ---------------------------------------------------------------------------

def test_config1_fp64_n16_vs_direct(su2):
    """N = 16, complex128, coefficients CN(0,1) seed 0, against the direct O(N^6) sum."""
    N = 16
    c = I.draw_coeffs(N, np.random.default_rng(0), "flat")
    f = T.inverse_separable(c, N)
    ref = T.forward_direct(f)
    _, (got,) = run_forward(su2, [f], "c128")
    assert rel(got, ref) < TOL64


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_forward_random_grid(su2, N, dtype):
    f = cast(I.draw_grid_gaussian((N, N, N), np.random.default_rng(1000 + N)), dtype)
    ref = T.forward_separable(f)
    _, (got,) = run_forward(su2, [f], dtype)
    assert rel(got, ref) < tol(dtype), rel(got, ref)


@pytest.mark.parametrize("dtype", ["c64"])
def test_forward_n128_bandlimited(su2, dtype):
    N = 128
    rng = np.random.default_rng(77)
    f = cast(I.draw_grid_gaussian((N, N, N), rng), dtype)
    # sampled pairs (the full O(N^4) oracle is slow at N = 128)
    _, (got,) = run_forward(su2, [f], dtype)
    from oracle import grid as G
    worst, scale = 0.0, 0.0
    pairs = [(0, 0), (126, 126), (-126, 126), (127, -127), (1, 1), (-37, 63), (50, -2), (-99, -99)]
    for n2, m2 in pairs:
        j0, vals = T.forward_pair(f, n2, m2)
        for i, v in enumerate(vals):
            worst = max(worst, abs(got[G.coeff_index(j0 + 2 * i, m2, n2)] - v))
            scale = max(scale, abs(v))
    assert worst / scale < TOL32


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_forward_batch(su2, dtype):
    N, B = 32, 3
    rng = np.random.default_rng(5)
    grids = [cast(I.draw_grid_gaussian((N, N, N), rng), dtype) for _ in range(B)]
    _, outs = run_forward(su2, grids, dtype)
    for g, o in zip(grids, outs):
        assert rel(o, T.forward_separable(g)) < tol(dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_forward_ragged(su2, dtype):
    Ns = [16, 64, 4, 32, 16, 8]
    rng = np.random.default_rng(6)
    grids = [cast(I.draw_grid_gaussian((n, n, n), rng), dtype) for n in Ns]
    _, outs = run_forward(su2, grids, dtype, Ns=Ns)
    for g, o in zip(grids, outs):
        assert rel(o, T.forward_separable(g)) < tol(dtype)


def test_forward_riemann_weights(su2):
    N = 16
    f = I.draw_grid_gaussian((N, N, N), np.random.default_rng(8))
    _, (got,) = run_forward(su2, [f], "c128", weights="riemann")
    assert rel(got, T.forward_separable(f, weights="riemann")) < TOL64


def test_constant_function(su2):
    N = 32
    f = np.ones((N, N, N), dtype=np.complex128)
    _, (got,) = run_forward(su2, [f], "c64")
    ref = T.forward_separable(f)
    assert abs(got[0] - 1.0) < 1e-6
    assert rel(got, ref) < TOL32


def test_config2_forward_and_inverse_n64(su2):
    """N = 64 complex64: coefficients CN(0,(1+l)^-2) seed 1, plus N(0, 0.01) grid noise."""
    N = 64
    rng = np.random.default_rng(1)
    c = I.draw_coeffs(N, rng, "inv2")
    f = T.inverse_separable(c, N) + I.draw_grid_noise((N, N, N), 0.01, rng)
    f = cast(f, "c64")
    plan, (got,) = run_forward(su2, [f], "c64")
    assert rel(got, T.forward_separable(f)) < TOL32
    # inverse of the (cast) coefficients
    c32 = cast(c, "c64")
    g = plan.inverse(to_dev(c32, "c64"))
    plan.sync_status()
    g = g.cpu().numpy().astype(np.complex128).reshape(N, N, N)
    assert rel(g, T.inverse_separable(c32, N)) < TOL32


# ---------------------------------------------------------------------------
# Inverse and adjoint
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("N", [4, 16, 32, 64])
def test_inverse(su2, N, dtype):
    c = cast(I.draw_coeffs(N, np.random.default_rng(200 + N)), dtype)
    plan = su2.Plan(N=N, batch=1, dtype=dtype)
    g = plan.inverse(to_dev(c, dtype))
    plan.sync_status()
    g = g.cpu().numpy().astype(np.complex128).reshape(N, N, N)
    assert rel(g, T.inverse_separable(c, N)) < tol(dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("N", [8, 32, 64])
def test_adjoint(su2, N, dtype):
    c = cast(I.draw_coeffs(N, np.random.default_rng(300 + N)), dtype)
    plan = su2.Plan(N=N, batch=1, dtype=dtype)
    g = plan.backward(to_dev(c, dtype))
    plan.sync_status()
    g = g.cpu().numpy().astype(np.complex128).reshape(N, N, N)
    assert rel(g, T.adjoint_separable(c, N)) < tol(dtype)


def test_inverse_ragged(su2):
    Ns = [32, 8, 16]
    rng = np.random.default_rng(9)
    cs = [cast(I.draw_coeffs(n, rng), "c64") for n in Ns]
    plan = su2.Plan(Ns=Ns, dtype="c64")
    g = plan.inverse(to_dev(np.concatenate(cs), "c64"))
    plan.sync_status()
    g = g.cpu().numpy().astype(np.complex128)
    for n, c, o in zip(Ns, cs, plan.grid_offsets):
        assert rel(g[o:o + n ** 3].reshape(n, n, n), T.inverse_separable(c, n)) < TOL32


def test_roundtrip_sector_fp64(su2):
    N = 32
    c = I.draw_coeffs(N, np.random.default_rng(10))
    two_l = I.packed_two_l(N)
    cs = np.where(two_l % 2 == 0, c, 0)
    plan = su2.Plan(N=N, batch=1, dtype="c128")
    back = plan.forward(plan.inverse(to_dev(cs, "c128")))
    plan.sync_status()
    back = back.cpu().numpy()
    sel = two_l % 2 == 0
    assert np.max(np.abs(back[sel] - cs[sel])) < 1e-12 * np.max(np.abs(cs))


def test_determinism(su2):
    N = 64
    f = I.draw_grid_gaussian((N, N, N), np.random.default_rng(11))
    plan = su2.Plan(N=N, batch=1, dtype="c64")
    x = to_dev(f, "c64")
    a = plan.forward(x).clone()
    b = plan.forward(x).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_rejects_bad_tensors(su2):
    plan = su2.Plan(N=16, batch=1, dtype="c64")
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(16 ** 3, dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(17, dtype=torch.complex64, device="cuda"))


# ---------------------------------------------------------------------------
# Tensor-core (split-BF16) contraction
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B", [1, 3])
def test_forward_tc_n64(su2, B):
    N = 64
    rng = np.random.default_rng(400 + B)
    grids = [cast(I.draw_grid_gaussian((N, N, N), rng), "c64") for _ in range(B)]
    _, outs = run_forward(su2, grids, "c64", algo="tc_bf16x3")
    for g, o in zip(grids, outs):
        assert rel(o, T.forward_separable(g)) < TOL32, rel(o, T.forward_separable(g))


def test_forward_tc_bandlimited_n64(su2):
    N = 64
    rng = np.random.default_rng(1)
    c = I.draw_coeffs(N, rng, "inv2")
    f = cast(T.inverse_separable(c, N) + I.draw_grid_noise((N, N, N), 0.01, rng), "c64")
    _, (got,) = run_forward(su2, [f], "c64", algo="tc_bf16x3")
    assert rel(got, T.forward_separable(f)) < TOL32


def test_forward_tc_ragged(su2):
    Ns = [64, 128, 64]
    rng = np.random.default_rng(12)
    grids = [cast(I.draw_grid_gaussian((n, n, n), rng), "c64") for n in Ns]
    _, outs = run_forward(su2, grids, "c64", Ns=Ns, algo="tc_bf16x3")
    from oracle import grid as G
    for n, g, o in zip(Ns, grids, outs):
        if n == 64:
            assert rel(o, T.forward_separable(g)) < TOL32
        else:
            worst = scale = 0.0
            for n2, m2 in [(0, 0), (126, -126), (127, 127), (-5, 3), (44, 44), (-1, -127)]:
                j0, vals = T.forward_pair(g, n2, m2)
                for i, v in enumerate(vals):
                    worst = max(worst, abs(o[G.coeff_index(j0 + 2 * i, m2, n2)] - v))
                    scale = max(scale, abs(v))
            assert worst / scale < TOL32


@pytest.mark.parametrize("algo", ["fp32", "tc_bf16x3"])
def test_full_size_n256_b64_sampled(su2, algo):
    """The benchmark's launch configuration (N = 256, 64 functions, complex64):
    4 seeded grids tiled over the 64 batch slots; sampled (m, n) pairs of every
    slot against the oracle's per-pair transform."""
    N, B = 256, 64
    rng = np.random.default_rng(2)
    base = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(4)]
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo=algo)
    x = torch.empty(B * N ** 3, dtype=torch.complex64, device="cuda")
    for b in range(B):
        x[b * N ** 3:(b + 1) * N ** 3].copy_(torch.from_numpy(base[b % 4].reshape(-1)))
    out = plan.forward(x)
    plan.sync_status()
    from oracle import grid as G
    pairs = [(0, 0), (254, 254), (-254, 254), (255, -255), (1, 1), (-77, 129), (30, -2), (-201, -201), (3, 255)]
    C = I.num_coeffs(N)
    ref = {}
    for gi in range(4):
        f64 = base[gi].astype(np.complex128)
        ref[gi] = {pq: T.forward_pair(f64, *pq) for pq in pairs}
    for b in range(0, B, 7):
        got = out[b * C:(b + 1) * C].cpu().numpy()
        worst = scale = 0.0
        for (n2, m2), (j0, vals) in ref[b % 4].items():
            for i, v in enumerate(vals):
                worst = max(worst, abs(got[G.coeff_index(j0 + 2 * i, m2, n2)] - v))
                scale = max(scale, abs(v))
        assert worst / scale < TOL32, (b, worst / scale)


def test_forward_tc_mixed_bandwidths(su2):
    """A tensor-core plan with bandwidths outside {64, 128, 256}: those groups
    take the FP32 contraction, the others the tensor cores."""
    Ns = [16, 64, 32, 128, 16]
    rng = np.random.default_rng(13)
    grids = [cast(I.draw_grid_gaussian((n, n, n), rng), "c64") for n in Ns]
    _, outs = run_forward(su2, grids, "c64", Ns=Ns, algo="tc_bf16x3")
    from oracle import grid as G
    for n, g, o in zip(Ns, grids, outs):
        if n <= 64:
            assert rel(o, T.forward_separable(g)) < TOL32, n
        else:
            worst = scale = 0.0
            for n2, m2 in [(0, 0), (126, -126), (127, 127), (-5, 3), (44, 44), (-1, -127)]:
                j0, vals = T.forward_pair(g, n2, m2)
                for i, v in enumerate(vals):
                    worst = max(worst, abs(o[G.coeff_index(j0 + 2 * i, m2, n2)] - v))
                    scale = max(scale, abs(v))
            assert worst / scale < TOL32


@pytest.mark.parametrize("algo", ["fp32", "tc_bf16x3"])
def test_inverse_n128_vs_oracle(su2, algo):
    """Synthesis at N = 128 (the two-phase inverse DFT) against the oracle,
    two functions (the second checks the per-function offsets)."""
    N = 128
    rng = np.random.default_rng(14)
    cs = [cast(I.draw_coeffs(N, rng, "inv1"), "c64") for _ in range(2)]
    plan = su2.Plan(N=N, batch=2, dtype="c64", algo=algo)
    g = plan.inverse(to_dev(np.concatenate(cs), "c64"))
    plan.sync_status()
    g = g.cpu().numpy().astype(np.complex128)
    for b in range(2):
        o = plan.grid_offsets[b]
        assert rel(g[o:o + N ** 3].reshape(N, N, N), T.inverse_separable(cs[b], N)) < TOL32, b


@pytest.mark.parametrize("N,B", [(128, 3), (256, 2), (512, 1)])
def test_roundtrip_and_adjoint_identity_large(su2, N, B):
    """Properties that hold at any size, for the two-phase inverse DFT and the
    fused transposed contraction: recovery within the sector of band-limited
    single-sector coefficients, forward(inverse(c)) = c there (on the paper's
    half domain the other sector receives leakage, so only the kept sector is
    compared), and <A f, g> = <f, A^H g>."""
    rng = np.random.default_rng(15 + N)
    plan = su2.Plan(N=N, batch=B, dtype="c64")
    C = I.num_coeffs(N)
    two_l = I.packed_two_l(N)
    cs, keep = [], []
    for b in range(B):
        c = I.draw_coeffs(N, rng, "inv1").astype(np.complex64)
        kept = (two_l % 2) == (b % 2)          # b even: integer l, b odd: half-integer l
        c[~kept] = 0
        cs.append(c)
        keep.append(torch.from_numpy(kept).cuda())
    c = torch.from_numpy(np.concatenate(cs)).cuda()
    grid = plan.inverse(c)
    back = plan.forward(grid)
    plan.sync_status()
    for b in range(B):
        cb, bb = c[b * C:(b + 1) * C][keep[b]], back[b * C:(b + 1) * C][keep[b]]
        d = (bb - cb).abs().max().item() / cb.abs().max().item()
        assert d < TOL32, (b, d)
    f = torch.randn(plan.grid_elems, dtype=torch.complex64, device="cuda")
    gg = torch.randn(plan.coeff_elems, dtype=torch.complex64, device="cuda")
    af = plan.forward(f)
    lhs = torch.vdot(af.to(torch.complex128), gg.to(torch.complex128))
    rhs = torch.vdot(f.to(torch.complex128), plan.backward(gg).to(torch.complex128))
    plan.sync_status()
    scale = (af.abs().double().norm() * gg.abs().double().norm()).item()
    assert abs((lhs - rhs).item()) < TOL32 * scale
