"""The differentiation workload at full size: batch 8 at N = 512, complex64
(1 GiB per grid), forward + hand-written adjoint through SU2FFT.

Full-size checks are ones the oracle can do one by one or properties that
hold at any size: sampled (m, n) pairs of every function against the oracle's
per-pair transform; the adjoint identity <A f, g> = <f, A^H g> on the whole
batch; the loss gradient through autograd equal to A^H[2 (2l+1)(A f - target)]
assembled from the library's own forward and adjoint.  The FP64 central
finite-difference check of the same autograd path runs at N = 8
(test_gpu_autograd.py)."""
import numpy as np
import pytest

import su2inputs as I
from oracle import grid as OG
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, B = 512, 8
TOL = 1e-5


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def batch():
    rng = np.random.default_rng(4)
    base = [I.draw_grid_gaussian((N, N, N), rng).astype(np.complex64) for _ in range(2)]
    x = torch.empty(B * N ** 3, dtype=torch.complex64, device="cuda")
    for b in range(B):
        x[b * N ** 3:(b + 1) * N ** 3].copy_(torch.from_numpy(base[b % 2].reshape(-1)))
    return base, x


def test_forward_n512_b8_sampled(su2, batch):
    base, x = batch
    plan = su2.Plan(N=N, batch=B, dtype="c64")
    out = plan.forward(x)
    plan.sync_status()
    pairs = [(0, 0), (510, 510), (-510, 510), (511, -511), (1, 1), (-77, 301), (300, -2), (3, 511)]
    C = I.num_coeffs(N)
    ref = {}
    for gi in range(2):
        f64 = base[gi].astype(np.complex128)
        ref[gi] = {pq: T.forward_pair(f64, *pq) for pq in pairs}
    for b in range(B):
        got = out[b * C:(b + 1) * C].cpu().numpy()
        worst = scale = 0.0
        for (n2, m2), (j0, vals) in ref[b % 2].items():
            for i, v in enumerate(vals):
                worst = max(worst, abs(got[OG.coeff_index(j0 + 2 * i, m2, n2)] - v))
                scale = max(scale, abs(v))
        assert worst / scale < TOL, (b, worst / scale)


def test_adjoint_identity_and_loss_gradient_n512_b8(su2, batch):
    _, x = batch
    plan = su2.Plan(N=N, batch=B, dtype="c64")
    C = I.num_coeffs(N)
    rng = np.random.default_rng(5)
    tgt = torch.empty(B * C, dtype=torch.complex64, device="cuda")
    for b in range(B):
        tgt[b * C:(b + 1) * C].copy_(torch.from_numpy(I.draw_coeffs(N, rng, "inv2").astype(np.complex64)))
    # adjoint identity on the whole batch (accumulated in FP64)
    fx = plan.forward(x)
    ag = plan.backward(tgt)
    plan.sync_status()
    lhs = torch.vdot(fx.to(torch.complex128), tgt.to(torch.complex128))
    rhs = torch.vdot(x.to(torch.complex128), ag.to(torch.complex128))
    scale = (fx.abs().double().norm() * tgt.abs().double().norm()).item()
    assert abs((lhs - rhs).item()) < TOL * scale
    # loss gradient through autograd
    wl = torch.from_numpy((I.packed_two_l(N) + 1).astype(np.float32)).cuda().repeat(B)
    xg = x.clone().requires_grad_(True)
    c = su2.SU2FFT.apply(xg, plan)
    loss = (wl * (c - tgt).abs() ** 2).sum()
    loss.backward()
    r = (2 * wl * (fx - tgt)).to(torch.complex64)
    g_ref = plan.backward(r)
    plan.sync_status()
    d = (xg.grad - g_ref).abs().max().item() / g_ref.abs().max().item()
    assert d < TOL, d
