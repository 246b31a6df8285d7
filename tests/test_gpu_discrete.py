"""Parity of the discrete (categorical) family (Sec. 4, 'Discrete') on the
CUDA path with the FP64 oracle: log-emission table, forward-backward,
symbol-count statistics, the M-step, a short fit and Viterbi, small and
large N, with the same tolerances as the other families."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import assert_params_close, check_fit_iterations, check_viterbi_fp64, check_viterbi_table_batch

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4
PARAM_RTOL = 1e-4
LENGTHS = [1, 2, 0, 37, 130, 9, 64, 65, 300]
CASES = [(2, 2), (3, 6), (16, 4), (64, 8)]


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


@pytest.fixture(scope="module")
def ctx(H):
    return H.Context(0)


def om(d):
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(),
                   {k: np.array(v, copy=True) for k, v in d["params"].items()})


def setup(H, ctx, N, K, lengths=LENGTHS, n_models=2, seed=0):
    models = synth.small_models("discrete", N, n_models, seed=1500 + seed + N + K, D=K)
    mid = np.arange(len(lengths)) % n_models
    values, offsets, mid = synth.make_batch(1600 + seed + N, models, lengths, mid)
    return models, values, offsets, mid, H.Model(ctx, models), H.Batch(values, offsets, mid)


@pytest.mark.parametrize("N,K", CASES)
def test_discrete_forward_backward(H, ctx, N, K):
    models, values, offsets, mid, model, batch = setup(H, ctx, N, K)
    lb = H.emission_logpdf(ctx, model, batch).cpu().numpy()
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    ll, gamma = ll.cpu().numpy(), gamma.cpu().numpy()
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        o = om(models[mid[s]])
        np.testing.assert_allclose(lb[offsets[s]:offsets[s + 1]], O.emission_logpdf(o, y), rtol=1e-6, atol=1e-6)
        fb = O.forward_backward(o, y)
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"]))
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL, rtol=0)


@pytest.mark.parametrize("N,K", CASES)
def test_discrete_estep_counts(H, ctx, N, K):
    models, values, offsets, mid, model, batch = setup(H, ctx, N, K, n_models=3, seed=1)
    stats, _ = H.estep_stats(ctx, model, batch)
    got = stats.get()
    off = 0
    for m, md in enumerate(models):
        o = om(md)
        g1, xi, ll, cnt = np.zeros(N), np.zeros((N, N)), 0.0, np.zeros((N, K))
        idx = [s for s in range(len(LENGTHS)) if mid[s] == m]
        for s in idx:
            y = values[offsets[s]:offsets[s + 1]]
            if len(y) == 0:
                continue
            fb = O.forward_backward(o, y)
            ll += fb["logL"]
            g1 += fb["gamma"][0]
            xi += fb["xi_sum"]
            for k in range(K):
                cnt[:, k] += fb["gamma"][y == k].sum(axis=0)
        ref = np.concatenate([[len(idx), ll], g1, xi.ravel(), cnt.ravel()])
        np.testing.assert_allclose(got[off:off + len(ref)], ref, rtol=2e-5, atol=2e-4)
        off += len(ref)


@pytest.mark.parametrize("N,K", CASES)
def test_discrete_mstep_and_fit(H, ctx, N, K):
    truth = synth.small_models("discrete", N, 1, seed=1700 + N, D=K)
    lengths = [400, 250, 1, 333, 128]
    values, offsets, mid = synth.make_batch(1701, truth, lengths, np.zeros(len(lengths), np.int32))
    rng = np.random.default_rng(10)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in init], values, offsets, mid)
    for g, r in zip(model.get(), ref):
        np.testing.assert_allclose(g["A"], r.A, rtol=PARAM_RTOL, atol=1e-6)
        np.testing.assert_allclose(g["params"]["p"], r.params["p"], rtol=PARAM_RTOL, atol=1e-6)
    model2 = H.Model(ctx, init)
    trace, (ref_models, ref_trace) = check_fit_iterations(H, ctx, model2, batch, values, offsets, mid, 4, atol=1e-6)
    np.testing.assert_allclose(trace[:, 0], ref_trace.sum(axis=1), rtol=LL_RTOL)
    assert_params_close(model2.get(), ref_models, rtol=PARAM_RTOL, atol=1e-6)


@pytest.mark.parametrize("N,K", CASES)
def test_discrete_viterbi(H, ctx, N, K):
    models, values, offsets, mid, model, batch = setup(H, ctx, N, K, seed=2)
    path, score = H.viterbi(ctx, model, batch)
    path, score = path.cpu().numpy(), score.cpu().numpy()
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            continue
        o = om(models[mid[s]])
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], o, y, where=s)
    # the decode is a function of the float32 table: bit-exact with the float32-mode oracle
    check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score)
