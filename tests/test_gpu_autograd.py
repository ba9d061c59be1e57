"""Differentiation through the library: SU2FFT (forward + hand-written adjoint)
against FP64 central finite differences of the GPU forward (torch gradcheck)
and against the oracle's gradient 2 A^H[(2l+1)(A f - target)]."""
import numpy as np
import pytest

import su2inputs as I
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def test_gradcheck_fp64_n8(su2):
    """The full Jacobian (every one of the 2 * 8^3 real inputs perturbed, every
    output's vector-Jacobian product), not one random projection."""
    N = 8
    plan = su2.Plan(N=N, batch=1, dtype="c128")
    g = I.draw_grid_gaussian((N, N, N), np.random.default_rng(3))
    x = torch.from_numpy(g.reshape(-1)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: su2.SU2FFT.apply(t, plan), (x,), eps=1e-6, atol=1e-7, rtol=1e-6,
                                    fast_mode=False)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 1e-5)])
def test_loss_gradient_matches_oracle(su2, dtype, tol):
    N = 8
    rng = np.random.default_rng(4)
    f = I.draw_grid_gaussian((N, N, N), rng)
    tgt = I.draw_coeffs(N, rng, "inv2")
    if dtype == "c64":
        f = f.astype(np.complex64).astype(np.complex128)
        tgt = tgt.astype(np.complex64).astype(np.complex128)
    L_ref, g_ref = T.loss_and_grad(f, tgt)
    plan = su2.Plan(N=N, batch=1, dtype=dtype)
    td = torch.complex128 if dtype == "c128" else torch.complex64
    x = torch.from_numpy(f.reshape(-1)).to(td).cuda().requires_grad_(True)
    t = torch.from_numpy(tgt).to(td).cuda()
    wl = torch.from_numpy((I.packed_two_l(N) + 1).astype(np.float64)).cuda()
    c = su2.SU2FFT.apply(x, plan)
    loss = (wl * (c - t).abs() ** 2).sum()
    loss.backward()
    g = x.grad.detach().cpu().numpy().astype(np.complex128).reshape(N, N, N)
    assert abs(loss.item() - L_ref) < tol * abs(L_ref) * 10
    assert np.max(np.abs(g - g_ref)) < tol * np.max(np.abs(g_ref))
