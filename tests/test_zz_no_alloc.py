"""su2_forward_noalloc: the forward transform for callers that cannot allocate
device memory when they transform (no allocator available in their code, a
memory budget fixed up front, or a steady-state loop that must not allocate).
It runs the same kernels as su2_forward but keeps the stage-1 planes in the
library's own fixed scratch array, so no workspace is passed.

Checked through the C ABI against su2_forward with a caller workspace, on two
calls in a row (the second call reuses the scratch the first one left behind,
and must leave the device's free memory unchanged), for uniform, ragged and
graph-recording plans, plus the size limit.  Named to be collected last.
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


@pytest.mark.parametrize("Ns,dtype,tol,graph", [([32, 32], "c64", 1e-5, False), ([64], "c64", 1e-5, False),
                                               ([16, 16, 16], "c128", 1e-12, False), ([32, 32], "c64", 1e-5, True),
                                               ([16, 32, 16], "c64", 1e-5, False)])
def test_noalloc_matches_workspace_path(su2, Ns, dtype, tol, graph):
    # graph=True: a plan that records su2_forward into a CUDA graph; the
    # allocation-free call still launches its kernels one by one.  [16, 32, 16]:
    # a ragged plan, whose bandwidth groups run on the plan's own streams and
    # keep their planes at disjoint offsets of the one scratch array.
    lib = su2.load()
    plan = su2.Plan(Ns=Ns, dtype=dtype, graph=graph)
    assert plan.workspace_bytes <= (4 << 20)
    td = torch.complex128 if dtype == "c128" else torch.complex64
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(sum(Ns))
    for call in range(2):
        g = np.zeros(plan.grid_elems, dtype=np.complex128)
        for n, o in zip(plan.Ns, plan.grid_offsets):
            g[o:o + n ** 3] = I.draw_grid_gaussian((n, n, n), rng).reshape(-1)
        grid = torch.from_numpy(g).to(td).cuda()
        ref = plan.forward(grid)
        out = torch.full((plan.coeff_elems,), float("nan"), dtype=td, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = lib.su2_forward_noalloc(plan._h, ctypes.c_void_p(grid.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream))
        assert st == 0, f"call {call}: status {st}"
        plan.sync_status()
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:
            # the first call may load kernel code (lazy module loading); the
            # second one must leave the device's free memory exactly as it was
            assert free_after == free_before, (free_before, free_after)
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
