"""Sharded forward transform (beta nodes split for stage 1, (s, m) rows for
stage 2) on one GPU: R ranks are run one after the other in this process and
the all-to-all is done by slicing, so only the library's two calls are
exercised.  Each plane value and each contraction is computed exactly as in
su2_forward, so the summed coefficients must equal su2_forward's bit for bit."""
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


@pytest.mark.parametrize("N,B,R", [(64, 3, 2), (64, 2, 4), (128, 2, 8), (256, 64, 2)])
def test_sharded_equals_forward(su2, N, B, R):
    from paper_2605_23923_gb300.sharded import partition
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo="tc_bf16x3")
    g = torch.randn(B * N ** 3, dtype=torch.complex64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(N + R))
    ref = plan.forward(g)
    g4 = g.view(B, N, N, N)
    parts = [partition(N, R, r) for r in range(R)]
    xs = []
    for (kb, nk, _, _) in parts:
        slab = g4[:, :, kb:kb + nk, :].contiguous().view(-1)
        xs.append(plan.forward_stage1_slab(kb, nk, slab).clone())
    total = torch.zeros_like(ref)
    for (_, nk, r0, nr) in parts:
        recv = torch.cat([x.view(2 * N, -1)[r0:r0 + nr].reshape(-1) for x in xs])
        total += plan.forward_stage2_rows(r0, nr, nk, recv)
    plan.sync_status()
    assert torch.equal(total, ref)


def test_sharded_argument_checks(su2):
    plan = su2.Plan(N=64, batch=1, dtype="c64", algo="tc_bf16x3")
    x = torch.zeros(2 * 64 * 64 * 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(su2.SU2Error):                 # nk not a multiple of 16
        plan.forward_stage2_rows(0, 1, 8, torch.zeros(64 * 64, dtype=torch.complex64, device="cuda"))
    with pytest.raises(su2.SU2Error):                 # beta range beyond N
        plan.forward_stage1_slab(60, 8, torch.zeros(64 * 8 * 64, dtype=torch.complex64, device="cuda"), out=x)
    fp32 = su2.Plan(N=64, batch=1, dtype="c64", algo="fp32")
    with pytest.raises(su2.SU2Error):                 # the sharded path is the tensor-core one
        fp32.forward_stage1_slab(0, 16, torch.zeros(64 * 16 * 64, dtype=torch.complex64, device="cuda"))
