"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (plan + autotuned chain widths): sampled sequences against the FP64
oracle one by one, and properties that hold at any size over the whole batch
(every gamma row sums to 1, the statistics' totals equal the sequence and
transition counts, the M-step keeps A row-stochastic)."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import check_viterbi_fp64

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


def om(d):
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(),
                   {k: np.array(v, copy=True) for k, v in d["params"].items()})


def stats_invariants(H, ctx, model, batch, models, offsets, mid, N):
    stats, _ = H.estep_stats(ctx, model, batch)
    rec = stats.get()
    fam_count = {"gamma": 4, "gauss": 3, "poisson": 2, "negbin": 3, "vonmises": 3, "student_t": 5,
                 "diag_gauss": None}
    off = 0
    lengths = np.diff(offsets)
    for m, md in enumerate(models):
        k = fam_count[md["family"]]
        size = 2 + N + N * N + N * k
        r = rec[off:off + size]
        off += size
        sel = mid == m
        assert r[0] == sel.sum()
        np.testing.assert_allclose(r[2:2 + N].sum(), sel.sum(), rtol=1e-6)            # sum_j gamma_1(j)
        xi = r[2 + N:2 + N + N * N].sum()                                              # sum of xi
        np.testing.assert_allclose(xi, np.maximum(lengths[sel] - 1, 0).sum(), rtol=1e-5)
        W = r[2 + N + N * N::k].sum()                                                  # sum of gamma
        np.testing.assert_allclose(W, lengths[sel].sum(), rtol=1e-5)
    return stats


def test_scale_full_size(H):
    """N = 16, 4096 x 2000, Gamma (the benchmark's default workload)."""
    truth, init, values, offsets, mid = synth.scale_workload("gamma")
    ctx = H.Context(0)
    model = H.Model(ctx, [init])
    batch = H.Batch(values, offsets, mid).make_plan(ctx, model)
    batch.autotune(ctx, model)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    # every gamma row of the 8.2M rows sums to 1
    rowsum = gamma.sum(dim=1)
    assert float((rowsum - 1).abs().max()) < 1e-4
    ll = ll.cpu().numpy()
    o = om(init)
    for s in (0, 1, 1023, 2048, 4095):
        y = values[offsets[s]:offsets[s + 1]]
        fb = O.forward_backward(o, y)
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * abs(fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]].cpu().numpy(), fb["gamma"], atol=GAMMA_ATOL)
    path, score = H.viterbi(ctx, model, batch)
    path, score = path.cpu().numpy(), score.cpu().numpy()
    for s in (0, 3000):
        y = values[offsets[s]:offsets[s + 1]]
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], o, y, where=("scale", s))
    stats = stats_invariants(H, ctx, model, batch, [init], offsets, mid, 16)
    H.mstep(ctx, model, stats, batch=batch)
    got = model.get()[0]
    np.testing.assert_allclose(got["A"].sum(axis=1), 1.0, rtol=1e-9)
    assert np.all(got["params"]["alpha"] > 0) and np.all(got["params"]["beta"] > 0)


def test_batching_full_size(H):
    """100k ragged sequences (lognormal lengths, 50-20000), N = 8, 1024 models
    of Gaussian / Poisson / negative-binomial / von Mises emissions."""
    truths, inits, values, offsets, mid = synth.batching_workload()
    ctx = H.Context(0)
    model = H.Model(ctx, inits)
    batch = H.Batch(values, offsets, mid).make_plan(ctx, model)
    batch.autotune(ctx, model)
    ll, _, _ = H.forward_backward(ctx, model, batch, want_gamma=False)
    ll = ll.cpu().numpy()
    lengths = np.diff(offsets)
    picks = [0, 1, int(np.argmax(lengths)), int(np.argmin(lengths)), 50000, 99999]
    for s in picks:
        fb = O.forward_backward(om(inits[mid[s]]), values[offsets[s]:offsets[s + 1]])
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"])), s
    stats = stats_invariants(H, ctx, model, batch, inits, offsets, mid, 8)
    H.mstep(ctx, model, stats, batch=batch)
    for g in model.get():
        np.testing.assert_allclose(g["A"].sum(axis=1), 1.0, rtol=1e-9)


def test_precision_full_size(H):
    """N = 512 (Dirichlet(0.1) rows), 1024 x 4096, diagonal Gaussian D = 32:
    the float32 path to the parity bar, the tensor path to its own bounds,
    on a sampled sequence's log-likelihood and on every gamma row."""
    from paper_2605_29208_gb300 import _lib
    truth, init, values, offsets, mid = synth.large_state_workload()
    ctx = H.Context(0)
    model = H.Model(ctx, [init])
    batch = H.Batch(values, offsets, mid, dim=values.shape[1]).make_plan(ctx, model)
    ll0, gamma, _ = H.forward_backward(ctx, model, batch)
    assert float((gamma.sum(dim=1) - 1).abs().max()) < 1e-4
    o = om(init)
    s = 517
    y = np.asarray(values[offsets[s]:offsets[s + 1]], np.float64)
    fb = O.forward_backward(o, y)              # the sampled sequence, element by element
    g0 = gamma[offsets[s]:offsets[s + 1]].cpu().numpy()
    np.testing.assert_allclose(g0, fb["gamma"], atol=GAMMA_ATOL)
    del gamma
    ctx.set_option(_lib.OPT_TENSOR_RECURRENCE, 1)
    ll1, gamma1, _ = H.forward_backward(ctx, model, batch)
    assert float((gamma1.sum(dim=1) - 1).abs().max()) < 1e-3
    g1 = gamma1[offsets[s]:offsets[s + 1]].cpu().numpy()
    # the FP16-operand path to its own stated bound
    assert float(np.abs(g1 - fb["gamma"]).max()) < 1e-3
    del gamma1
    ll0, ll1 = ll0.cpu().numpy(), ll1.cpu().numpy()
    ref = fb["logL"]
    assert abs(ll0[s] - ref) <= LL_RTOL * abs(ref)
    assert abs(ll1[s] - ref) <= 5e-5 * abs(ref)
    assert np.all(np.abs(ll1 - ll0) <= 5e-5 * np.abs(ll0))
    # the statistics of the whole batch on the tensor path: totals equal the
    # sequence, transition and row counts, the M-step keeps A stochastic
    stats, _ = H.estep_stats(ctx, model, batch)
    rec = stats.get()
    N = 512
    n_seq, g1s, xi = rec[0], rec[2:2 + N], rec[2 + N:2 + N + N * N]
    W = rec[2 + N + N * N:].reshape(N, -1)[:, 0]
    assert n_seq == 1024
    assert abs(g1s.sum() - 1024) < 1e-2
    assert abs(xi.sum() - 1024 * 4095) < 1e-3 * 1024 * 4095
    assert abs(W.sum() - 1024 * 4096) < 1e-3 * 1024 * 4096
    H.mstep(ctx, model, stats, batch=batch)
    np.testing.assert_allclose(model.get()[0]["A"].sum(axis=1), 1.0, rtol=1e-9)
