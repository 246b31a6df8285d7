"""Failure detection without a GPU fault: a bounded device wait that runs
out turns into an error status the host reads, and the context stays
usable.  hmm_ctx_wait_selftest waits, with the wait the tensor-core kernels
use, on an mbarrier phase that nothing completes; a limit of about a
millisecond makes it expire."""
import ctypes as C
import time

import numpy as np
import pytest

from paper_2605_29208_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


def test_expired_wait_reports_timeout_and_context_survives(H):
    ctx = H.Context(0)
    assert ctx.status() == 0
    waited = C.c_int64(0)
    limit = 2_000_000                       # ~1 ms of SM cycles
    t0 = time.perf_counter()
    H.check(ctx.lib.hmm_ctx_wait_selftest(ctx.h, limit, C.byref(waited), None))
    dt = time.perf_counter() - t0
    assert waited.value >= limit            # it waited the whole limit ...
    assert dt < 5.0                         # ... and came back
    assert ctx.status() == 5                # HMM_E_TIMEOUT, then cleared
    assert ctx.status() == 0
    # the context still computes
    models = synth.small_models("gauss", 3, 1, seed=2)
    values, offsets, mid = synth.make_batch(4, models, [50, 20], [0, 0])
    ll, _, _ = H.forward_backward(ctx, H.Model(ctx, models), H.Batch(values, offsets, mid))
    assert np.all(np.isfinite(ll.cpu().numpy()))
    assert ctx.status() == 0


def test_wait_selftest_rejects_bad_limits(H):
    ctx = H.Context(0)
    for bad in (0, -5, 1 << 40):
        assert ctx.lib.hmm_ctx_wait_selftest(ctx.h, bad, None, None) == 1
