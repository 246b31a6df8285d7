"""Data-parallel exchange on one GPU: two ranks, each a host thread with its
own context, model and statistics, run hmm_estep_stats and hmm_mstep on
their halves of a batch with the library's all-reduce hook installed
(hmm_stats_set_allreduce).  The hook combines the two ranks' device records
(float64 sums, int32 minima of the support keys, and the sums of every
Newton data pass); the host waits for both ranks at each call, so no kernel
waits on another.  After the M-step both ranks must hold bit-identical
models equal to the M-step of the whole batch in one process, for all 17
families (Sec. 4: every statistic is a sum over sequences, a minimum /
maximum over rows or a per-pass sum).  Also an empty shard, and the sizes
and ops of the calls."""
import threading

import numpy as np
import pytest

from paper_2605_29208_gb300 import synth

pytestmark = pytest.mark.gpu

FAMILIES = ["gauss", "poisson", "gamma", "beta", "weibull", "negbin", "student_t", "vonmises",
            "diag_gauss", "full_gauss", "discrete", "lognormal", "exponential", "rayleigh", "uniform",
            "chisq", "pareto"]
DIM = {"diag_gauss": 3, "full_gauss": 3, "discrete": 5}
# Newton iterations stop on a relative step; summation order alone moves the
# result by far less than this
RTOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


class PairReduce:
    """All-reduce between two host threads of this process: each call waits
    (on the host) for the other rank's call with the same size and op, then
    both receive the combination of the two records."""

    def __init__(self):
        self.barrier = threading.Barrier(2, timeout=120)
        self.slots = [None, None]
        self.result = None

    def for_rank(self, rank):
        def reduce(t, op, stream):
            import torch
            torch.cuda.synchronize()
            self.slots[rank] = (t, op)
            self.barrier.wait()
            if rank == 0:
                (a, oa), (b, ob) = self.slots
                assert oa == ob and a.numel() == b.numel() and a.dtype == b.dtype
                self.result = a + b if op == 0 else torch.minimum(a, b)
                torch.cuda.synchronize()
            self.barrier.wait()
            t.copy_(self.result)
            torch.cuda.synchronize()
            self.barrier.wait()
        return reduce


def make_case(family, N=4, seed=0):
    D = DIM.get(family, 1)
    truth = synth.small_models(family, N, 2, seed=4100 + seed + FAMILIES.index(family), D=D)
    lengths = [120, 7, 1, 333, 64, 250, 2, 90, 45, 300]
    mid = np.arange(len(lengths)) % 2
    values, offsets, mid = synth.make_batch(4200 + seed, truth, lengths, mid)
    rng = np.random.default_rng(seed + 5)
    init = [synth.perturb(rng, t) for t in truth]
    bdim = D if family in ("diag_gauss", "full_gauss") else 1
    return init, np.asarray(values).reshape(-1, bdim) if bdim > 1 else values, offsets, mid, bdim


def sub_batch(values, offsets, mid, lo, hi):
    o = offsets[lo:hi + 1] - offsets[lo]
    return values[offsets[lo]:offsets[hi]], o, mid[lo:hi]


def run_rank(H, init, values, offsets, mid, bdim, reduce, out, rank):
    from paper_2605_29208_gb300 import parallel
    try:
        ctx = H.Context(0)
        model = H.Model(ctx, init)
        batch = H.Batch(values, offsets, mid, dim=bdim)
        stats = H.Stats(ctx, model)
        ex = parallel.Exchange(stats, reduce=reduce)
        H.estep_stats(ctx, model, batch, stats=stats)
        H.mstep(ctx, model, stats, batch=batch)
        ex.close()
        assert ex.error is None, ex.error
        out[rank] = (model.get(), list(ex.calls), stats.get())
    except BaseException as e:                     # surfaced by the main thread
        out[rank] = e


def two_ranks(H, init, values, offsets, mid, bdim, split):
    pr = PairReduce()
    parts = [sub_batch(values, offsets, mid, 0, split), sub_batch(values, offsets, mid, split, len(mid))]
    out = [None, None]
    th = [threading.Thread(target=run_rank, args=(H, init, *parts[r], bdim, pr.for_rank(r), out, r))
          for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    for r in range(2):
        if isinstance(out[r], BaseException):
            raise out[r]
    return out


def full_batch(H, init, values, offsets, mid, bdim):
    ctx = H.Context(0)
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid, dim=bdim)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    return model.get(), stats.get()


def assert_models_close(a, b, rtol):
    for x, y in zip(a, b):
        np.testing.assert_allclose(x["pi"], y["pi"], rtol=rtol, atol=1e-15)
        np.testing.assert_allclose(x["A"], y["A"], rtol=rtol, atol=1e-15)
        for k in y["params"]:
            np.testing.assert_allclose(x["params"][k], y["params"][k], rtol=rtol, atol=1e-14, err_msg=k)


def assert_models_equal(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x["pi"], y["pi"])
        np.testing.assert_array_equal(x["A"], y["A"])
        for k in y["params"]:
            np.testing.assert_array_equal(x["params"][k], y["params"][k], err_msg=k)


@pytest.mark.parametrize("family", FAMILIES)
def test_two_rank_exchange_equals_full_batch(H, family):
    init, values, offsets, mid, bdim = make_case(family)
    (m0, calls0, st0), (m1, calls1, st1) = two_ranks(H, init, values, offsets, mid, bdim, split=4)
    assert calls0 == calls1
    assert_models_equal(m0, m1)
    ref, ref_st = full_batch(H, init, values, offsets, mid, bdim)
    # the combined statistics are the whole batch's (sums in another order)
    np.testing.assert_allclose(st0, ref_st, rtol=1e-12, atol=1e-9)
    assert_models_close(m0, ref, RTOL)
    n_pass = sum(1 for n, op in calls0[1:] if op == 0 and n == 2 * 4 * 3)
    if family in ("weibull", "negbin"):
        assert n_pass >= 2                          # one exchange per Newton data pass
    if family in ("uniform", "pareto"):
        assert any(op == 1 for _, op in calls0)     # support minima


@pytest.mark.parametrize("family", ["gamma", "negbin", "pareto", "full_gauss"])
def test_empty_shard_takes_part_in_the_exchange(H, family):
    init, values, offsets, mid, bdim = make_case(family, seed=3)
    (m0, calls0, _), (m1, calls1, _) = two_ranks(H, init, values, offsets, mid, bdim, split=0)
    assert calls0 == calls1
    assert_models_equal(m0, m1)
    ref, _ = full_batch(H, init, values, offsets, mid, bdim)
    assert_models_close(m0, ref, RTOL)
