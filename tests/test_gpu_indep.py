"""Independent-components emissions (Sec. 4.5) on the GPU against the FP64
oracle: densities, forward-backward, the per-component weighted sums, one
M-step, fits checked per iteration, and Viterbi (float64 oracle, and bit
for bit with the float32-mode oracle on the device's own float32 table).
Component sets: the paper's Gamma + von Mises example, and the other
supported scalar families, at small and large state counts."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import (GAMMA_ATOL, LL_RTOL, PARAM_RTOL, assert_params_close, check_fit_iterations, check_viterbi_fp64,
                    check_viterbi_table_batch, om)

pytestmark = pytest.mark.gpu

CASES = [
    (("gamma", "vonmises"), 2),
    (("gamma", "vonmises"), 5),
    (("gauss", "poisson", "beta"), 3),
    (("student_t", "lognormal", "exponential", "rayleigh", "chisq"), 4),
    (("gamma", "vonmises", "gauss"), 40),
]
IDS = ["+".join(c) + f"-N{n}" for c, n in CASES]
LENGTHS = [1, 2, 0, 37, 130, 9, 300, 64, 65]


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


def setup(H, ctx, comps, N, lengths=LENGTHS, n_models=2, seed=0, init=False):
    truth = synth.indep_models(list(comps), N, n_models, seed=3300 + seed + N + len(comps))
    mid = np.arange(len(lengths)) % n_models
    values, offsets, mid = synth.make_batch(3400 + seed + N, truth, lengths, mid)
    values = np.asarray(values).reshape(-1, len(comps))
    models = truth
    if init:
        rng = np.random.default_rng(seed + 11)
        models = [synth.perturb(rng, t) for t in truth]
    return models, values, offsets, mid, H.Model(ctx, models), H.Batch(values, offsets, mid, dim=len(comps))


def oracle_indep_stats(models, values, offsets, mid):
    """Canonical statistics of hmm_stats_get from the oracle's occupancies:
    per model n_seq, sum logL, gamma_1 sums, xi sums, then per state W and
    each component's weighted sums."""
    out = []
    for m, model in enumerate(models):
        o = om(model)
        N = len(model["pi"])
        idx = [s for s in range(len(offsets) - 1) if mid[s] == m and offsets[s + 1] > offsets[s]]
        g1, xi, ll, Ws, Ys = np.zeros(N), np.zeros((N, N)), 0.0, [], []
        for s in idx:
            y = values[offsets[s]:offsets[s + 1]]
            fb = O.forward_backward(o, y)
            ll += fb["logL"]
            g1 += fb["gamma"][0]
            xi += fb["xi_sum"]
            Ws.append(fb["gamma"])
            Ys.append(y)
        W, Y = np.concatenate(Ws), np.concatenate(Ys)
        n_seq = sum(1 for s in range(len(offsets) - 1) if mid[s] == m)
        rec = [n_seq, ll, *g1, *xi.ravel()]
        for j in range(N):
            w = W[:, j]
            rec.append(w.sum())
            for d, f in enumerate(model["components"]):
                y = Y[:, d]
                with np.errstate(all="ignore"):
                    ly = np.log(np.where(y > 0, y, 1.0))
                if f in ("gauss",):
                    rec += [(w * y).sum(), (w * y * y).sum()]
                elif f in ("poisson", "exponential"):
                    rec += [(w * y).sum()]
                elif f == "gamma":
                    rec += [(w * y).sum(), (w * ly).sum(), (w * y * y).sum()]
                elif f == "beta":
                    rec += [(w * y).sum(), (w * y * y).sum(), (w * ly).sum(), (w * np.log1p(-y)).sum()]
                elif f == "student_t":
                    p = model["params"]
                    u = O.student_t_utilde(y, p[f"d{d}.mu"][j], p[f"d{d}.sigma2"][j], p[f"d{d}.nu"][j])
                    rec += [(w * u).sum(), (w * u * y).sum(), (w * u * y * y).sum(), (w * (np.log(u) - u)).sum()]
                elif f == "vonmises":
                    rec += [(w * np.cos(y)).sum(), (w * np.sin(y)).sum()]
                elif f == "lognormal":
                    rec += [(w * ly).sum(), (w * ly * ly).sum()]
                elif f == "rayleigh":
                    rec += [(w * y * y).sum()]
                elif f == "chisq":
                    rec += [(w * ly).sum()]
        out.append(np.array(rec))
    return np.concatenate(out)


@pytest.mark.parametrize("comps,N", CASES, ids=IDS)
def test_indep_emission_and_forward_backward(H, ctx, comps, N):
    models, values, offsets, mid, model, batch = setup(H, ctx, comps, N)
    lb = H.emission_logpdf(ctx, model, batch).cpu().numpy()
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    ll, gamma = ll.cpu().numpy(), gamma.cpu().numpy()
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        o = om(models[mid[s]])
        np.testing.assert_allclose(lb[offsets[s]:offsets[s + 1]], O.emission_logpdf(o, y), rtol=2e-5, atol=2e-4)
        fb = O.forward_backward(o, y)
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"])), (s, ll[s], fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL)


@pytest.mark.parametrize("comps,N", CASES, ids=IDS)
def test_indep_estep_stats(H, ctx, comps, N):
    models, values, offsets, mid, model, batch = setup(H, ctx, comps, N, seed=1)
    stats, _ = H.estep_stats(ctx, model, batch)
    got = stats.get()
    ref = oracle_indep_stats(models, values, offsets, mid)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=2e-4)


@pytest.mark.parametrize("comps,N", CASES, ids=IDS)
def test_indep_mstep_and_fit(H, ctx, comps, N):
    lengths = [400, 250, 1, 333, 128, 90]
    models, values, offsets, mid, model, batch = setup(H, ctx, comps, N, lengths=lengths, seed=2, init=True)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in models], values, offsets, mid)
    assert_params_close(model.get(), ref, rtol=PARAM_RTOL, atol=1e-6)
    model2 = H.Model(ctx, models)
    trace, (ref_models, ref_trace) = check_fit_iterations(H, ctx, model2, batch, values, offsets, mid, 4, atol=1e-6)
    np.testing.assert_allclose(trace.sum(axis=1), ref_trace.sum(axis=1), rtol=LL_RTOL)
    assert_params_close(model2.get(), ref_models, rtol=PARAM_RTOL, atol=1e-6)


@pytest.mark.parametrize("comps,N", CASES, ids=IDS)
def test_indep_viterbi(H, ctx, comps, N):
    models, values, offsets, mid, model, batch = setup(H, ctx, comps, N, seed=3)
    path, score = H.viterbi(ctx, model, batch)
    path, score = path.cpu().numpy(), score.cpu().numpy()
    for s in range(len(LENGTHS)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            continue
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], om(models[mid[s]]), y, where=(comps, N, s))
    check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score)


def test_indep_rejects_unsupported_components(H, ctx):
    from paper_2605_29208_gb300 import HmmError
    m = synth.indep_models(["gamma", "vonmises"], 3, 1, seed=1)[0]
    m["components"] = ["gamma", "weibull"]
    m["params"]["d1.k"] = np.ones(3)
    m["params"]["d1.lam"] = np.ones(3)
    with pytest.raises(HmmError) as e:
        H.Model(ctx, [m])
    assert "UNSUPPORTED" in str(e.value)
