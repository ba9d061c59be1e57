"""The workspace needs no initialisation: every transform gives bit-identical
results whether the workspace starts zeroed or filled with 0xFF bytes (NaN
in every float lane).  Parts of the stage-1 planes that belong to no
coefficient (the integer sector's Nyquist row and column) are never written by
the synthesis / adjoint contraction, so a kernel that scaled them by zero
instead of leaving them out would turn such bytes into NaN."""
import numpy as np
import pytest

import su2inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


CASES = [(16, 2, "c64", "fp32"), (64, 3, "c64", "fp32"), (64, 2, "c64", "tc_bf16x3"), (128, 2, "c64", "fp32"),
         (256, 2, "c64", "fp32"), (256, 1, "c64", "tc_bf16x3"), (512, 1, "c64", "fp32"), (16, 2, "c128", "fp64"),
         (64, 1, "c128", "fp64")]


@pytest.mark.parametrize("N,B,dtype,algo", CASES)
def test_results_do_not_depend_on_workspace_content(su2, N, B, dtype, algo):
    plan = su2.Plan(N=N, batch=B, dtype=dtype, algo=algo)
    td = plan.torch_dtype
    rng = np.random.default_rng(N + B)
    g = np.concatenate([I.draw_grid_gaussian((N, N, N), rng).reshape(-1) for _ in range(B)])
    c = np.concatenate([I.draw_coeffs(N, rng, "inv1") for _ in range(B)])
    grid = torch.from_numpy(g).to(td).cuda()
    coef = torch.from_numpy(c).to(td).cuda()
    res = {}
    for fill in (0x00, 0xFF):
        ws = torch.full((max(plan.workspace_bytes, 16),), fill, dtype=torch.uint8, device="cuda")
        fwd = plan.forward(grid, ws=ws).clone()
        ws.fill_(fill)
        inv = plan.inverse(coef, ws=ws).clone()
        ws.fill_(fill)
        adj = plan.backward(coef, ws=ws).clone()
        plan.sync_status()
        res[fill] = (fwd, inv, adj)
        del ws
    for name, a, b in zip(("forward", "inverse", "backward"), res[0x00], res[0xFF]):
        assert torch.isfinite(torch.view_as_real(a)).all(), name
        assert torch.equal(a, b), name
    plan.close()
