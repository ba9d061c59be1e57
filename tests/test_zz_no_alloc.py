"""su2_forward_noalloc: the forward transform for callers that cannot allocate
device memory when they transform (no allocator available in their code, a
memory budget fixed up front, or a steady-state loop that must not allocate).
It runs the same kernels as su2_forward but keeps the stage-1 planes in the
library's own fixed scratch array, so no workspace is passed.

Checked through the C ABI against su2_forward with a caller workspace, on two
calls in a row (the second call reuses the scratch the first one left behind),
plus the size limit.  Named to be collected last.
"""
import ctypes

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


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("N,B,dtype,tol,graph", [(32, 2, "c64", 1e-5, False), (64, 1, "c64", 1e-5, False),
                                                 (16, 3, "c128", 1e-12, False), (32, 2, "c64", 1e-5, True)])
def test_noalloc_matches_workspace_path(su2, N, B, dtype, tol, graph):
    # graph=True: a plan that records su2_forward into a CUDA graph; the
    # allocation-free call still launches its kernels one by one
    lib = su2.load()
    plan = su2.Plan(N=N, batch=B, dtype=dtype, graph=graph)
    assert plan.workspace_bytes <= (4 << 20)
    td = torch.complex128 if dtype == "c128" else torch.complex64
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(N + B)
    for call in range(2):
        g = np.concatenate([I.draw_grid_gaussian((N, N, N), rng).reshape(-1) for _ in range(B)])
        grid = torch.from_numpy(g).to(td).cuda()
        ref = plan.forward(grid)
        out = torch.full((plan.coeff_elems,), float("nan"), dtype=td, device="cuda")
        st = lib.su2_forward_noalloc(plan._h, ctypes.c_void_p(grid.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream))
        assert st == 0, f"call {call}: status {st}"
        plan.sync_status()
        assert torch.isfinite(out.real).all() and torch.isfinite(out.imag).all()
        assert _rel(out, ref) < tol, (call, _rel(out, ref))


def test_noalloc_rejects_plans_beyond_the_scratch_size(su2):
    lib = su2.load()
    plan = su2.Plan(N=128, batch=1, dtype="c64")           # 32 MiB of planes > 4 MiB
    grid = torch.zeros(plan.grid_elems, dtype=torch.complex64, device="cuda")
    out = torch.zeros(plan.coeff_elems, dtype=torch.complex64, device="cuda")
    st = lib.su2_forward_noalloc(plan._h, ctypes.c_void_p(grid.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 6                                         # SU2_ERR_WORKSPACE
