"""Parity of the multivariate families (Sec. 4.5: diagonal Gaussian, Eq.
20-21; full-covariance Gaussian, Eq. 22-24) on the CUDA path with the FP64
oracle: emission log-densities, forward-backward, statistics, the M-step,
a short fit and Viterbi.  Tolerances as for the scalar families."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import check_fit_iterations, check_viterbi_fp64, check_viterbi_table_batch

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4
PARAM_RTOL = 1e-4

LENGTHS = [1, 2, 0, 33, 64, 65, 200, 257]
CASES = [("diag_gauss", 2, 3), ("diag_gauss", 5, 4), ("full_gauss", 3, 3), ("full_gauss", 4, 8),
         ("diag_gauss", 16, 2), ("full_gauss", 8, 5)]


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


def setup(H, ctx, family, N, D, lengths=LENGTHS, n_models=2, seed=0):
    models = synth.small_models(family, N, n_models, seed=200 + seed + N + D, D=D)
    mid = np.arange(len(lengths)) % n_models
    values, offsets, mid = synth.make_batch(300 + seed + N, models, lengths, mid)
    values = values.reshape(-1, D)
    return models, values, offsets, mid, H.Model(ctx, models), H.Batch(values, offsets, mid, dim=D)


@pytest.mark.parametrize("family,N,D", CASES)
def test_mv_emission(H, ctx, family, N, D):
    models, values, offsets, mid, model, batch = setup(H, ctx, family, N, D)
    lb = H.emission_logpdf(ctx, model, batch).cpu().numpy()
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            continue
        ref = O.emission_logpdf(om(models[mid[s]]), y.astype(np.float64))
        np.testing.assert_allclose(lb[offsets[s]:offsets[s + 1]], ref, rtol=2e-5, atol=2e-4)


@pytest.mark.parametrize("family,N,D", CASES)
def test_mv_forward_backward(H, ctx, family, N, D):
    models, values, offsets, mid, model, batch = setup(H, ctx, family, N, D)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    ll = ll.cpu().numpy()
    gamma = gamma.cpu().numpy()
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]].astype(np.float64)
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        fb = O.forward_backward(om(models[mid[s]]), y)
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"])), (s, ll[s], fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL, rtol=0)


def oracle_canonical_mv(models, values, offsets, mid):
    """hmm_stats_get's layout for the multivariate families: per model
    [n_seq, sum logL, sum gamma_1, sum xi, then per state W, sum g y,
    sum g y_d^2 (diagonal) or sum g y y^T (full)], from oracle occupancies."""
    out = []
    for m, model in enumerate(models):
        o = om(model)
        N = len(model["pi"])
        idx = [s for s in range(len(offsets) - 1) if mid[s] == m]
        g1, xi, ll = np.zeros(N), np.zeros((N, N)), 0.0
        Ws, Ys = [], []
        for s in idx:
            y = values[offsets[s]:offsets[s + 1]].astype(np.float64)
            if len(y) == 0:
                continue
            fb = O.forward_backward(o, y)
            ll += fb["logL"]
            g1 += fb["gamma"][0]
            xi += fb["xi_sum"]
            Ws.append(fb["gamma"])
            Ys.append(y)
        W, Y = np.concatenate(Ws), np.concatenate(Ys)
        cols = []
        for j in range(N):
            w = W[:, j]
            second = (w[:, None] * Y * Y).sum(0) if model["family"] == "diag_gauss" else \
                np.einsum("t,td,te->de", w, Y, Y).ravel()
            cols.append(np.concatenate([[w.sum()], (w[:, None] * Y).sum(0), second]))
        out.append(np.concatenate([[len(idx), ll], g1, xi.ravel(), np.ravel(cols)]))
    return np.concatenate(out)


@pytest.mark.parametrize("family,N,D", CASES)
def test_mv_estep_stats(H, ctx, family, N, D):
    models, values, offsets, mid, model, batch = setup(H, ctx, family, N, D, n_models=3)
    stats, _ = H.estep_stats(ctx, model, batch)
    got = stats.get()
    ref = oracle_canonical_mv(models, values, offsets, mid)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=2e-4)


def assert_params_close(got_models, ref_models, rtol):
    for g, r in zip(got_models, ref_models):
        np.testing.assert_allclose(g["pi"], r.pi, rtol=rtol, atol=1e-6)
        np.testing.assert_allclose(g["A"], r.A, rtol=rtol, atol=1e-6)
        for k, v in r.params.items():
            np.testing.assert_allclose(g["params"][k], v, rtol=rtol, atol=1e-6, err_msg=f"{r.family}.{k}")


@pytest.mark.parametrize("family,N,D", CASES)
def test_mv_mstep(H, ctx, family, N, D):
    truth = synth.small_models(family, N, 2, seed=400 + N + D, D=D)
    lengths = [400, 250, 1, 333, 128, 90]
    values, offsets, mid = synth.make_batch(17 + N, truth, lengths, np.arange(len(lengths)) % 2)
    values = values.reshape(-1, D)
    rng = np.random.default_rng(5)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid, dim=D)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in init], values.astype(np.float64), offsets, mid)
    assert_params_close(model.get(), ref, PARAM_RTOL)


@pytest.mark.parametrize("family,N,D", [("diag_gauss", 4, 3), ("full_gauss", 3, 4)])
def test_mv_fit(H, ctx, family, N, D):
    truth = synth.small_models(family, N, 1, seed=500 + N + D, D=D)
    lengths = [500, 300, 211, 64]
    values, offsets, mid = synth.make_batch(23, truth, lengths, np.zeros(len(lengths), np.int32))
    values = values.reshape(-1, D)
    rng = np.random.default_rng(6)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid, dim=D)
    trace, (ref_models, ref_trace) = check_fit_iterations(H, ctx, model, batch, values.astype(np.float64), offsets,
                                                          mid, 5)
    np.testing.assert_allclose(trace[:, 0], ref_trace.sum(axis=1), rtol=LL_RTOL)
    assert_params_close(model.get(), ref_models, PARAM_RTOL)
    assert np.all(np.diff(trace[:, 0]) >= -1e-6 * np.abs(trace[:, 0]).max())


@pytest.mark.parametrize("family,N,D", CASES)
def test_mv_viterbi_vs_fp64(H, ctx, family, N, D):
    models, values, offsets, mid, model, batch = setup(H, ctx, family, N, D)
    path, score = H.viterbi(ctx, model, batch)
    path = path.cpu().numpy()
    score = score.cpu().numpy()
    # the internal emission table and the caller's table give the same result
    lb = H.emission_logpdf(ctx, model, batch)
    path2, score2 = H.viterbi(ctx, model, batch, logb=lb)
    np.testing.assert_array_equal(path, path2.cpu().numpy())
    np.testing.assert_array_equal(score, score2.cpu().numpy())
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]].astype(np.float64)
        if len(y) == 0:
            continue
        o = om(models[mid[s]])
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], o, y, where=(family, N, D, s))
    check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score)


def test_mv_not_positive_definite(H, ctx):
    """A covariance that is not positive definite gives density 0: the
    state's log b is -inf and the state never carries occupancy."""
    models = synth.small_models("full_gauss", 3, 1, seed=9, D=2)
    models[0]["params"]["cov"][1] = np.array([[1.0, 2.0], [2.0, 1.0]])
    values, offsets, mid = synth.make_batch(3, synth.small_models("full_gauss", 3, 1, seed=9, D=2), [50, 20],
                                            np.zeros(2, np.int32))
    values = values.reshape(-1, 2)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid, dim=2)
    lb = H.emission_logpdf(ctx, model, batch).cpu().numpy()
    assert np.all(np.isneginf(lb[:, 1]))
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    assert np.all(np.isfinite(ll.cpu().numpy()))
    assert np.all(gamma.cpu().numpy()[:, 1] == 0.0)


def test_mv_mixed_diag_and_full(H, ctx):
    """One model set holding both multivariate families (records of the
    diagonal states are padded to the full layout)."""
    D, N = 3, 4
    models = (synth.small_models("diag_gauss", N, 1, seed=41, D=D)
              + synth.small_models("full_gauss", N, 1, seed=42, D=D))
    lengths = [300, 1, 120, 257, 64]
    mid = np.arange(len(lengths)) % 2
    values, offsets, mid = synth.make_batch(29, models, lengths, mid)
    values = values.reshape(-1, D)
    rng = np.random.default_rng(8)
    init = [synth.perturb(rng, t) for t in models]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid, dim=D)
    stats, _ = H.estep_stats(ctx, model, batch)
    np.testing.assert_allclose(stats.get(), oracle_canonical_mv(init, values, offsets, mid), rtol=2e-5, atol=2e-4)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in init], values.astype(np.float64), offsets, mid)
    assert_params_close(model.get(), ref, PARAM_RTOL)


def test_mv_scalar_mix_rejected(H, ctx):
    models = synth.small_models("diag_gauss", 2, 1, seed=1, D=1) + synth.small_models("gauss", 2, 1, seed=2)
    with pytest.raises(Exception):
        H.Model(ctx, models)
