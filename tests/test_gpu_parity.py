"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs.  Tolerances (float32 device arithmetic):
per-sequence logL 1e-5 relative, occupancies 1e-4 absolute, M-step
parameters 1e-4 relative, Viterbi paths bit-identical to the float32-mode
oracle on a shared float32 log-emission table."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import check_fit_iterations, check_viterbi_fp32, check_viterbi_fp64

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4
PARAM_RTOL = 1e-4

SCALAR = ("gauss", "poisson", "gamma", "beta", "weibull", "negbin", "student_t", "vonmises")


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
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(), {k: np.array(v, copy=True) for k, v in d["params"].items()})


def ragged_batch(models, lengths, seed):
    mid = np.arange(len(lengths)) % len(models)
    return synth.make_batch(seed, models, lengths, mid)


LENGTHS = [1, 2, 3, 0, 7, 64, 65, 130, 257, 5, 300, 33]


def check_ll(got, ref, where=None):
    ref = np.asarray(ref)
    bad = np.abs(got - ref) > LL_RTOL * np.maximum(np.abs(ref), 1.0)
    assert not bad.any(), (where, np.nonzero(bad)[0], got[bad], ref[bad])


@pytest.mark.parametrize("family", SCALAR)
@pytest.mark.parametrize("N", [1, 3, 8, 16])
def test_forward_backward_parity(H, ctx, family, N):
    models = synth.small_models(family, N, 2, seed=100 + N)
    values, offsets, mid = ragged_batch(models, LENGTHS, seed=7 + N)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    ll, gamma, path = H.forward_backward(ctx, model, batch, want_path=True)
    ll = ll.cpu().numpy()
    gamma = gamma.cpu().numpy()
    path = path.cpu().numpy()
    oms = [om(m) for m in models]
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        fb = O.forward_backward(oms[mid[s]], y)
        check_ll(np.array([ll[s]]), np.array([fb["logL"]]), s)
        g = gamma[offsets[s]:offsets[s + 1]]
        np.testing.assert_allclose(g, fb["gamma"], atol=GAMMA_ATOL, rtol=0)
        # posterior decoding: equal wherever the oracle's best state is clear
        ref_path = O.posterior_decode(fb["gamma"])
        srt = np.sort(fb["gamma"], axis=1)
        clear = (srt[:, -1] - srt[:, -2] > 2 * GAMMA_ATOL) if N > 1 else np.ones(len(y), bool)
        np.testing.assert_array_equal(path[offsets[s]:offsets[s + 1]][clear], ref_path[clear])


@pytest.mark.parametrize("N", [2, 5, 16, 32])
def test_forward_backward_table_mode(H, ctx, N):
    """Emissions from a float32 log b table (the path used by the
    multivariate families): same recursions, table shared with the oracle."""
    rng = np.random.default_rng(N)
    models = synth.small_models("gauss", N, 1, seed=N)
    lengths = [1, 2, 9, 100, 401]
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    logb = rng.normal(-3, 2, (offsets[-1], N)).astype(np.float32)
    values = np.zeros(offsets[-1])
    mid = np.zeros(len(lengths), np.int32)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    import torch
    tlogb = torch.as_tensor(logb).cuda()
    ll, gamma, _ = H.forward_backward(ctx, model, batch, logb=tlogb)
    ll = ll.cpu().numpy()
    gamma = gamma.cpu().numpy()
    m = om(models[0])
    for s in range(len(lengths)):
        lb = logb[offsets[s]:offsets[s + 1]].astype(np.float64)
        fb = O.forward_backward_logb(np.log(m.pi), np.log(m.A), lb)
        check_ll(np.array([ll[s]]), np.array([fb["logL"]]), s)
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL)


def oracle_canonical_stats(models, values, offsets, mid):
    """The canonical sums the C ABI reports (hmm_stats_get), from the
    oracle's occupancies."""
    out = []
    for m, model in enumerate(models):
        o = om(model)
        N = len(model["pi"])
        idx = [s for s in range(len(offsets) - 1) if mid[s] == m]
        g1 = np.zeros(N)
        xi = np.zeros((N, N))
        fam = np.zeros((N, 0)).tolist()
        rows_w, rows_y, ll = [], [], 0.0
        for s in idx:
            y = values[offsets[s]:offsets[s + 1]]
            if len(y) == 0:
                continue
            fb = O.forward_backward(o, y)
            ll += fb["logL"]
            g1 += fb["gamma"][0]
            xi += fb["xi_sum"]
            rows_w.append(fb["gamma"])
            rows_y.append(y)
        W = np.concatenate(rows_w)
        Y = np.concatenate(rows_y)
        f = model["family"]
        cols = []
        for j in range(N):
            w = W[:, j]
            if f == "gauss":
                cols.append([w.sum(), (w * Y).sum(), (w * Y * Y).sum()])
            elif f == "poisson":
                cols.append([w.sum(), (w * Y).sum()])
            elif f == "gamma":
                cols.append([w.sum(), (w * Y).sum(), (w * np.log(Y)).sum(), (w * Y * Y).sum()])
            elif f == "beta":
                cols.append([w.sum(), (w * Y).sum(), (w * Y * Y).sum(), (w * np.log(Y)).sum(),
                             (w * np.log1p(-Y)).sum()])
            elif f == "student_t":
                p = model["params"]
                u = O.student_t_utilde(Y, p["mu"][j], p["sigma2"][j], p["nu"][j])
                cols.append([w.sum(), (w * u).sum(), (w * u * Y).sum(), (w * u * Y * Y).sum(),
                             (w * (np.log(u) - u)).sum()])
            elif f == "vonmises":
                cols.append([w.sum(), (w * np.cos(Y)).sum(), (w * np.sin(Y)).sum()])
            elif f == "weibull":
                cols.append([w.sum(), (w * np.log(Y)).sum(), (w * np.log(Y) ** 2).sum()])
            elif f == "negbin":
                cols.append([w.sum(), (w * Y).sum(), (w * Y * Y).sum()])
        out.append(np.concatenate([[len(idx), ll], g1, xi.ravel(), np.ravel(cols)]))
    return np.concatenate(out)


@pytest.mark.parametrize("family", SCALAR)
def test_estep_stats_parity(H, ctx, family):
    N = 4
    models = synth.small_models(family, N, 3, seed=11)
    values, offsets, mid = ragged_batch(models, [50, 3, 200, 120, 1, 77, 310, 64, 2], seed=5)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    stats, ll = H.estep_stats(ctx, model, batch)
    got = stats.get()
    ref = oracle_canonical_stats(models, values, offsets, mid)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-4)


def assert_params_close(got_models, ref_models, rtol=PARAM_RTOL):
    for g, r in zip(got_models, ref_models):
        np.testing.assert_allclose(g["pi"], r.pi, rtol=rtol, atol=1e-6)
        np.testing.assert_allclose(g["A"], r.A, rtol=rtol, atol=1e-6)
        for k, v in r.params.items():
            gv = g["params"][k]
            if r.family == "vonmises" and k == "mu":
                np.testing.assert_allclose(np.angle(np.exp(1j * (gv - v))), 0, atol=rtol)
            else:
                np.testing.assert_allclose(gv, v, rtol=rtol, atol=1e-7, err_msg=f"{r.family}.{k}")


@pytest.mark.parametrize("family", SCALAR)
def test_mstep_parity(H, ctx, family):
    N = 3
    truth = synth.small_models(family, N, 2, seed=21)
    values, offsets, mid = ragged_batch(truth, [400, 250, 1, 333, 128, 90], seed=9)
    rng = np.random.default_rng(3)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    got = model.get()
    ref, _ = O.em_iteration([om(m) for m in init], values, offsets, mid)
    assert_params_close(got, ref)


@pytest.mark.parametrize("family", ["gauss", "gamma", "student_t", "weibull", "negbin", "vonmises"])
def test_fit_parity(H, ctx, family):
    N = 4
    truth = synth.small_models(family, N, 1, seed=31)
    values, offsets, mid = ragged_batch(truth, [500, 300, 211, 64], seed=13)
    rng = np.random.default_rng(4)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid)
    trace, (ref_models, ref_trace) = check_fit_iterations(H, ctx, model, batch, values, offsets, mid, 5)
    # the compounded five iterations from the same start
    np.testing.assert_allclose(trace[:, 0], ref_trace.sum(axis=1), rtol=LL_RTOL)
    assert_params_close(model.get(), ref_models, rtol=PARAM_RTOL)
    # EM monotonicity on the device trace
    assert np.all(np.diff(trace[:, 0]) >= -1e-6 * np.abs(trace[:, 0]).max())


@pytest.mark.parametrize("N", [2, 3, 8, 16, 32])
def test_viterbi_bit_exact_table(H, ctx, N):
    import torch
    rng = np.random.default_rng(50 + N)
    models = synth.small_models("gauss", N, 1, seed=N, conc=0.5)
    lengths = [1, 2, 5, 64, 65, 129, 700]
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    logb = rng.normal(-2, 2, (offsets[-1], N)).astype(np.float32)
    # a few exact ties to exercise the tie rule
    logb[10:20] = np.round(logb[10:20])
    mid = np.zeros(len(lengths), np.int32)
    model = H.Model(ctx, models)
    batch = H.Batch(np.zeros(offsets[-1]), offsets, mid)
    path, score = H.viterbi(ctx, model, batch, logb=torch.as_tensor(logb).cuda())
    path = path.cpu().numpy()
    score = score.cpu().numpy()
    m = models[0]
    lpi = np.log(m["pi"]).astype(np.float32)
    lA = np.log(m["A"]).astype(np.float32)
    for s in range(len(lengths)):
        check_viterbi_fp32(path[offsets[s]:offsets[s + 1]], score[s], lpi, lA, logb[offsets[s]:offsets[s + 1]], N,
                           where=s)


@pytest.mark.parametrize("family", SCALAR)
def test_viterbi_vs_fp64(H, ctx, family):
    N = 5
    models = synth.small_models(family, N, 2, seed=61)
    values, offsets, mid = ragged_batch(models, [1, 2, 40, 200, 301, 77], seed=17)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    path, score = H.viterbi(ctx, model, batch)
    path = path.cpu().numpy()
    score = score.cpu().numpy()
    for s in range(len(offsets) - 1):
        y = values[offsets[s]:offsets[s + 1]]
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], om(models[mid[s]]), y, where=(family, s))


@pytest.mark.parametrize("family", SCALAR)
def test_emission_logpdf(H, ctx, family):
    models = synth.small_models(family, 6, 2, seed=71)
    values, offsets, mid = ragged_batch(models, [1, 50, 133], seed=19)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    lb = H.emission_logpdf(ctx, model, batch).cpu().numpy()
    for s in range(3):
        ref = O.emission_logpdf(om(models[mid[s]]), values[offsets[s]:offsets[s + 1]])
        np.testing.assert_allclose(lb[offsets[s]:offsets[s + 1]], ref, rtol=2e-5, atol=2e-4)


def test_zero_probability_sequence(H, ctx):
    models = synth.small_models("gamma", 3, 1, seed=3)
    values = np.array([1.0, 2.0, -1.0, 3.0, 0.5, 0.7])
    offsets = np.array([0, 4, 6], np.int64)
    mid = np.zeros(2, np.int32)
    model = H.Model(ctx, models)
    ll, gamma, _ = H.forward_backward(ctx, model, H.Batch(values, offsets, mid))
    ll = ll.cpu().numpy()
    assert ll[0] == -np.inf
    ref = O.forward_backward(om(models[0]), values[4:6])["logL"]
    check_ll(ll[1:], np.array([ref]))


def test_batching_mixed_families_ragged(H, ctx):
    """The batching workload at reduced size: ragged lognormal lengths, 24
    models of N = 8 states with Gaussian / Poisson / negative-binomial / von
    Mises emissions in one persistent launch; per-sequence logL and one EM
    iteration (all models) against the oracle."""
    truths, inits, values, offsets, mid = synth.batching_workload(
        n_seq=600, n_models=24, N=8, seed=77, median=100, tmin=10, tmax=1500)
    model = H.Model(ctx, inits)
    batch = H.Batch(values, offsets, mid).make_plan(ctx, model)
    ll, _, _ = H.forward_backward(ctx, model, batch, want_gamma=False)
    ll = ll.cpu().numpy()
    oms = [om(m) for m in inits]
    for s in range(0, 600, 7):
        fb = O.forward_backward(oms[mid[s]], values[offsets[s]:offsets[s + 1]])
        check_ll(np.array([ll[s]]), np.array([fb["logL"]]), s)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration(oms, values, offsets, mid)
    assert_params_close(model.get(), ref)


def test_autotune_keeps_results(H, ctx):
    """The autotuner only changes chain widths: log-likelihoods before and
    after tuning agree with each other and with the oracle."""
    truths, inits, values, offsets, mid = synth.batching_workload(
        n_seq=300, n_models=8, N=8, seed=78, median=80, tmin=5, tmax=3000)
    model = H.Model(ctx, inits)
    batch = H.Batch(values, offsets, mid).make_plan(ctx, model)
    ll0, _, _ = H.forward_backward(ctx, model, batch, want_gamma=False)
    ms = batch.autotune(ctx, model)
    assert ms[0] > 0 and ms[1] > 0
    ll1, _, _ = H.forward_backward(ctx, model, batch, want_gamma=False)
    ll0, ll1 = ll0.cpu().numpy(), ll1.cpu().numpy()
    np.testing.assert_allclose(ll1, ll0, rtol=2e-6, atol=1e-6)
    oms = [om(m) for m in inits]
    for s in range(0, 300, 17):
        fb = O.forward_backward(oms[mid[s]], values[offsets[s]:offsets[s + 1]])
        check_ll(np.array([ll1[s]]), np.array([fb["logL"]]), s)


def test_length_one_sequences_after_other_work(H, ctx):
    """A chain whose first step is in phase 2 (the forward chain of a length-1
    sequence) must not read a stale previous-vector buffer into xi: after a
    large launch has left arbitrary shared memory behind, the statistics of
    length-1 sequences are finite and their transition sums are zero."""
    models = synth.small_models("gamma", 16, 1, seed=5)
    v0, o0, m0 = synth.make_batch(5, models, [3000] * 64, np.zeros(64, np.int32))
    model = H.Model(ctx, models)
    H.forward_backward(ctx, model, H.Batch(v0, o0, m0))
    values, offsets, mid = synth.make_batch(6, models, [1] * 40, np.zeros(40, np.int32))
    stats, ll = H.estep_stats(ctx, model, H.Batch(values, offsets, mid))
    rec = stats.get()
    assert np.all(np.isfinite(rec))
    N = 16
    assert np.all(rec[2 + N:2 + N + N * N] == 0.0)
    fb = [O.forward_backward(om(models[0]), values[offsets[s]:offsets[s + 1]])["logL"] for s in range(40)]
    check_ll(ll.cpu().numpy(), np.array(fb))


def test_negbin_mstep_with_counts_above_the_histogram(H, ctx):
    """Negative-binomial states whose counts straddle the histogram range
    (means 20 and 700): the M-step's Newton sums combine the weighted
    histogram of the small counts with the data pass over the large ones."""
    rng = np.random.default_rng(5)
    r = np.array([5.0, 30.0])
    mean = np.array([20.0, 700.0])
    truth = [synth.make_model("negbin", np.array([0.5, 0.5]), np.array([[0.9, 0.1], [0.2, 0.8]]),
                              r=r, p=r / (r + mean))]
    values, offsets, mid = synth.make_batch(6, truth, [400, 250, 31, 500], [0, 0, 0, 0])
    assert (values >= 512).any() and (values < 512).any()
    init = [synth.perturb(rng, truth[0])]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in init], values, offsets, mid)
    assert_params_close(model.get(), ref)
