"""su2_forward_pipelined (host-resident batches streamed through the device)
gives the same coefficients as su2_forward on the same grids: uniform batches
that take several upload chunks, a ragged plan (several groups, coefficient
blocks not adjacent within a group), complex128, and two calls in a row on
one stream with different data (the second call's uploads overlap the first
call's stage 2 and downloads)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


def _pinned(n, dtype, gen):
    h = torch.empty(n, dtype=dtype, pin_memory=True)
    h.copy_(torch.randn(n, dtype=dtype, generator=gen))
    return h


def _reference(plan, host_grid):
    return plan.forward(host_grid.cuda()).cpu()


@pytest.mark.parametrize("N,B,algo", [(256, 10, "tc_bf16x3"), (128, 3, "fp32")])
def test_pipelined_matches_forward(su2, N, B, algo):
    gen = torch.Generator().manual_seed(600 + N)
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo=algo)
    hg = _pinned(plan.grid_elems, torch.complex64, gen)
    ref = _reference(plan, hg)
    stream = torch.cuda.current_stream()
    out = plan.forward_pipelined(hg, stream=stream)
    stream.synchronize()
    plan.sync_status()
    assert torch.equal(out, ref)


def test_pipelined_ragged(su2):
    Ns = [16, 64, 32, 64, 16, 128, 32]
    gen = torch.Generator().manual_seed(610)
    plan = su2.Plan(Ns=Ns, dtype="c64", algo="tc_bf16x3")
    hg = _pinned(plan.grid_elems, torch.complex64, gen)
    ref = _reference(plan, hg)
    out = plan.forward_pipelined(hg)
    torch.cuda.synchronize()
    plan.sync_status()
    assert torch.equal(out, ref)


def test_pipelined_c128(su2):
    gen = torch.Generator().manual_seed(620)
    plan = su2.Plan(N=16, batch=3, dtype="c128", algo="fp64")
    hg = _pinned(plan.grid_elems, torch.complex128, gen)
    ref = _reference(plan, hg)
    out = plan.forward_pipelined(hg)
    torch.cuda.synchronize()
    plan.sync_status()
    assert torch.equal(out, ref)


def test_pipelined_two_calls_in_a_row(su2):
    N, B = 256, 9
    gen = torch.Generator().manual_seed(630)
    plan = su2.Plan(N=N, batch=B, dtype="c64", algo="tc_bf16x3")
    h1 = _pinned(plan.grid_elems, torch.complex64, gen)
    h2 = _pinned(plan.grid_elems, torch.complex64, gen)
    r1, r2 = _reference(plan, h1), _reference(plan, h2)
    dev = torch.device("cuda")
    dg = torch.empty(plan.grid_elems, dtype=torch.complex64, device=dev)
    dc = torch.empty(plan.coeff_elems, dtype=torch.complex64, device=dev)
    o1 = torch.empty(plan.coeff_elems, dtype=torch.complex64, pin_memory=True)
    o2 = torch.empty(plan.coeff_elems, dtype=torch.complex64, pin_memory=True)
    stream = torch.cuda.current_stream()
    plan.forward_pipelined(h1, o1, dg, dc, stream=stream)
    plan.forward_pipelined(h2, o2, dg, dc, stream=stream)
    stream.synchronize()
    plan.sync_status()
    assert torch.equal(o1, r1) and torch.equal(o2, r2)
