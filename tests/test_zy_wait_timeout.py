"""Failure detection without a GPU fault: a kernel wait that runs out.

Every wait in the library's kernels is bounded.  When one runs out, it
latches MELT_ERR_TIMEOUT in the basis and lets its kernel finish.
melt_diag_wait_timeout launches a wait on a barrier that nothing arrives
on.  The test checks that the host reads the status once, after about the
bound, and that the context and the basis keep working.  The file sorts
last, so it runs after every other GPU test.
"""
import time

import numpy as np
import pytest

from paper_2606_01009_gb300 import inputs as G
from tests.helpers import gpu_features

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def melt():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_01009_gb300 import melt as m
    return m


def test_bounded_wait_reports_timeout_and_context_survives(melt):
    import torch
    fe = melt.Frontend(precision="bf16")
    clips = [G.rich_clip(4, i, 20000) for i in range(2)]
    before = gpu_features(fe, clips)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    melt.melt_diag_wait_timeout(fe.handle)
    with pytest.raises(melt.MeltError) as ei:
        fe.sync()
    dt = time.perf_counter() - t0
    assert ei.value.status == melt.MELT_ERR_TIMEOUT
    assert 0.5 < dt < 30.0, dt  # the wait's bound is 1 s of GPU time
    fe.sync()  # reported once, then cleared
    after = gpu_features(fe, clips)
    assert np.array_equal(before, after)
    fe.close()
