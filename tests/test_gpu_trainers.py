"""MAP Baum-Welch and Viterbi training (the trainers the paper names,
Sec. 5.6, in the readings the oracle states) on the GPU against the FP64
oracle: the MAP M-step and fit per iteration; the Viterbi-training E-step
(paths, scores, hard statistics), its M-step and fit per iteration, for
closed-form, Newton, data-pass, table and large-N families.  The data have
well-separated states, so the float32 and float64 decoders agree on every
path (checked) and the hard statistics can be compared."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import LL_RTOL, PARAM_RTOL, assert_params_close, check_viterbi_fp64, om

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


@pytest.fixture(scope="module")
def ctx(H):
    return H.Context(0)


def separated(family, N, seed, n_models=2):
    """Models whose states emit far apart, sticky transitions."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_models):
        A = 0.85 * np.eye(N) + 0.15 * rng.dirichlet(np.ones(N), size=N)
        pi = rng.dirichlet(np.ones(N))
        if family == "gauss":
            p = dict(mu=8.0 * np.arange(N) + rng.normal(0, 0.3, N), sigma2=rng.uniform(0.5, 1.5, N))
        elif family == "gamma":
            p = dict(alpha=20.0 * (1 + np.arange(N)), beta=np.full(N, 2.0) + rng.uniform(0, 0.2, N))
        elif family == "negbin":
            r = rng.uniform(20, 40, N)
            mean = 30.0 * (1 + np.arange(N))
            p = dict(r=r, p=r / (r + mean))
        elif family == "discrete":
            K = 2 * N
            pk = np.full((N, K), 0.02)
            for j in range(N):
                pk[j, 2 * j:2 * j + 2] = 1.0
            p = dict(p=pk / pk.sum(1, keepdims=True))
        out.append(synth.make_model(family, pi, A, **p))
    return out


def batch_of(H, models, seed, lengths=(300, 1, 250, 120, 77, 200)):
    mid = np.arange(len(lengths)) % len(models)
    values, offsets, mid = synth.make_batch(seed, models, list(lengths), mid)
    return values, offsets, mid, H.Batch(values, offsets, mid)


@pytest.mark.parametrize("family", ["gauss", "gamma", "negbin"])
def test_map_mstep_and_fit(H, ctx, family):
    truth = synth.small_models(family, 4, 2, seed=77)
    values, offsets, mid, batch = batch_of(H, truth, 78)
    rng = np.random.default_rng(79)
    init = [synth.perturb(rng, t) for t in truth]
    opts = H.mstep_opts(dirichlet_A=2.5, dirichlet_pi=3.0)
    model = H.Model(ctx, init)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch, opts=opts)
    ref, _ = O.em_iteration([om(m) for m in init], values, offsets, mid, alpha_A=2.5, alpha_pi=3.0)
    assert_params_close(model.get(), ref, rtol=PARAM_RTOL)
    # fits, iteration by iteration
    model2 = H.Model(ctx, init)
    for k in range(3):
        before = [om(m) for m in model2.get()]
        tr, done = H.fit(ctx, model2, batch, n_iter=1, opts=opts)
        ref, ll = O.em_iteration(before, values, offsets, mid, alpha_A=2.5, alpha_pi=3.0)
        np.testing.assert_allclose(tr[0], [ll[mid == m].sum() for m in range(2)], rtol=LL_RTOL)
        assert_params_close(model2.get(), ref, rtol=PARAM_RTOL)


def hard_canonical(models, values, offsets, mid):
    """Canonical statistics of the Viterbi paths from the oracle (gauss
    family sums)."""
    out = []
    for m, res in enumerate(O.viterbi_estep([om(x) for x in models], values, offsets, mid)):
        N = len(models[m]["pi"])
        W = np.concatenate(res["W"])
        Y = np.concatenate(res["Y"])
        rec = [res["n_seq"], sum(res["score"]), *res["gamma1_sum"], *res["xi_sum"].ravel()]
        for j in range(N):
            w = W[:, j]
            rec += [w.sum(), (w * Y).sum(), (w * Y * Y).sum()]
        out.append(np.array(rec))
    return np.concatenate(out)


@pytest.mark.parametrize("family,N", [("gauss", 3), ("gauss", 40), ("gamma", 4), ("negbin", 3), ("discrete", 3)])
def test_viterbi_training(H, ctx, family, N):
    truth = separated(family, N, seed=90 + N)
    values, offsets, mid, batch = batch_of(H, truth, 91 + N)
    init = [dict(t, params={k: v.copy() for k, v in t["params"].items()}) for t in truth]
    rng = np.random.default_rng(92)
    for m in init:                       # a start near the truth keeps the paths clear
        m["A"] = 0.9 * m["A"] + 0.1 / N
        for k, v in m["params"].items():
            if family != "discrete":
                m["params"][k] = v * rng.uniform(0.97, 1.03, v.shape)
    model = H.Model(ctx, init)
    stats, score = H.estep_viterbi(ctx, model, batch)
    score = score.cpu().numpy()
    res = O.viterbi_estep([om(m) for m in init], values, offsets, mid)
    path, _ = H.viterbi(ctx, model, batch)
    path = path.cpu().numpy()
    for m, r in enumerate(res):
        for s, q, sc in zip(r["seq"], r["path"], r["score"]):
            np.testing.assert_array_equal(path[offsets[s]:offsets[s + 1]], q)
            assert abs(score[s] - sc) <= LL_RTOL * max(1.0, abs(sc))
    if family == "gauss":
        np.testing.assert_allclose(stats.get(), hard_canonical(init, values, offsets, mid), rtol=2e-5, atol=2e-4)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.viterbi_train_iteration([om(m) for m in init], values, offsets, mid)
    assert_params_close(model.get(), ref, rtol=PARAM_RTOL)
    # fit with the Viterbi trainer, iteration by iteration; the objective never decreases
    model2 = H.Model(ctx, init)
    obj = []
    for k in range(3):
        before = [om(m) for m in model2.get()]
        # the paths of this iteration: equal to the float64 decoder's, else a
        # logged near-tie, after which the two trajectories may part
        p2, s2 = H.viterbi(ctx, model2, batch)
        p2, s2 = p2.cpu().numpy(), s2.cpu().numpy()
        tie = False
        for s in range(len(offsets) - 1):
            q, _ = O.viterbi(before[mid[s]], values[offsets[s]:offsets[s + 1]])
            if not np.array_equal(p2[offsets[s]:offsets[s + 1]], q):
                check_viterbi_fp64(p2[offsets[s]:offsets[s + 1]], s2[s], before[mid[s]],
                                   values[offsets[s]:offsets[s + 1]], where=("viterbi training", k, s))
                tie = True
        if tie:
            break
        tr, done = H.fit(ctx, model2, batch, n_iter=1, trainer="viterbi")
        ref, sc = O.viterbi_train_iteration(before, values, offsets, mid)
        np.testing.assert_allclose(tr[0], [sc[mid == m].sum() for m in range(len(init))], rtol=LL_RTOL)
        assert_params_close(model2.get(), ref, rtol=PARAM_RTOL)
        obj.append(tr[0].sum())
    assert len(obj) >= 2 and np.all(np.diff(obj) >= -1e-6 * abs(obj[0]))
