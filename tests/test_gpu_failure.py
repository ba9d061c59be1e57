"""Failure detection without a GPU fault: a kernel whose bounded wait can never
complete (a counter nothing increments, an mbarrier nothing arrives on) gives
up after about a second, the host reads SU2_ERR_TIMEOUT from su2_sync_status,
and the same context then runs a transform correctly."""
import time

import numpy as np
import pytest

import su2inputs as I
from oracle import transform as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SU2_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def su2():
    import paper_2605_23923_gb300 as m
    from paper_2605_23923_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_times_out_and_context_survives(su2, kind):
    N = 16
    plan = su2.Plan(N=N, batch=1, dtype="c64", algo="fp32")
    t0 = time.time()
    plan.selftest_bounded_wait(kind)
    with pytest.raises(su2.SU2Error) as ei:
        plan.sync_status()
    assert ei.value.status == SU2_ERR_TIMEOUT
    assert 0.2 < time.time() - t0 < 30.0                 # gave up after its limit, not at once
    plan.sync_status()                                    # the word was cleared
    f = I.draw_grid_gaussian((N, N, N), np.random.default_rng(7)).astype(np.complex64)
    got = plan.forward(torch.from_numpy(f.reshape(-1)).cuda()).cpu().numpy()
    plan.sync_status()
    ref = T.forward_separable(f.astype(np.complex128))
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-5


def test_selftest_rejects_unknown_kind(su2):
    plan = su2.Plan(N=16, batch=1, dtype="c64")
    with pytest.raises(su2.SU2Error):
        plan.selftest_bounded_wait(2)
