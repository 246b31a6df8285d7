"""Pins of the oracle's further scalar families (Sec. 4.1 log-normal,
exponential, Rayleigh, uniform; Sec. 4.2 chi-squared and Pareto) against
things other than the oracle itself:

* every log-density against scipy.stats (and -inf outside the support);
* every closed-form or 1-D M-step against a numerical maximiser of the
  weighted log-likelihood of Eq. 6 (scipy.optimize from a distant start);
* chi-squared against its score equation and scipy.stats.chi2.fit;
* the support reading of the Uniform / Pareto min and max: the rows with
  gamma_t(j) > 0 (float64 forward-backward) are the rows b_j(y_t) > 0;
* EM on each family never lowers the log-likelihood."""
import numpy as np
import pytest
from scipy import optimize, stats

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth

FAMS = ["lognormal", "exponential", "rayleigh", "uniform", "chisq", "pareto"]


def model(f, **params):
    N = len(next(iter(params.values())))
    return O.Model(f, np.full(N, 1.0 / N), np.full((N, N), 1.0 / N),
                   {k: np.asarray(v, np.float64) for k, v in params.items()})


def test_densities_match_scipy():
    y = np.array([-1.0, 0.0, 0.3, 1.0, 2.5, 7.0])
    cases = [
        (model("lognormal", mu=[0.2, -1.0], sigma2=[0.5, 2.0]),
         lambda j, p: stats.lognorm(s=np.sqrt(p["sigma2"][j]), scale=np.exp(p["mu"][j]))),
        (model("exponential", lam=[0.5, 3.0]), lambda j, p: stats.expon(scale=1 / p["lam"][j])),
        (model("rayleigh", sigma2=[0.7, 4.0]), lambda j, p: stats.rayleigh(scale=np.sqrt(p["sigma2"][j]))),
        (model("uniform", a=[-1.0, 0.3], b=[1.0, 2.5]),
         lambda j, p: stats.uniform(loc=p["a"][j], scale=p["b"][j] - p["a"][j])),
        (model("chisq", nu=[1.0, 5.5]), lambda j, p: stats.chi2(df=p["nu"][j])),
        (model("pareto", xm=[0.3, 2.0], alpha=[1.5, 4.0]),
         lambda j, p: stats.pareto(b=p["alpha"][j], scale=p["xm"][j])),
    ]
    for m, dist in cases:
        got = O.emission_logpdf(m, y)
        for j in range(2):
            ref = dist(j, m.params).logpdf(y)
            if m.family == "chisq":
                # reading: support y > 0 (at y = 0 the density is +inf for nu < 2)
                ref = np.where(y > 0, ref, -np.inf)
            # the closed uniform interval: scipy's density is positive at both ends too
            np.testing.assert_allclose(got[:, j], ref, rtol=1e-12, atol=1e-12, err_msg=m.family)


def weighted_data(f, seed=0, n=400):
    rng = np.random.default_rng(seed)
    truth = synth.random_params(rng, f, 1)
    d = dict(family=f, params=truth)
    y = synth.sample_emissions(rng, d, np.zeros(n, np.int64))
    w = rng.uniform(0.05, 1.0, n)
    return y, w, {k: v[0] for k, v in truth.items()}


def neg_q(f, w, y):
    def fn(theta):
        p = dict(zip(synth.PARAM_NAMES[f], theta))
        m = model(f, **{k: [v] for k, v in p.items()})
        lb = O.emission_logpdf(m, y)[:, 0]
        val = -np.sum(w * lb)
        return val if np.isfinite(val) else 1e300
    return fn


@pytest.mark.parametrize("f", ["lognormal", "exponential", "rayleigh", "chisq"])
def test_mstep_is_the_weighted_maximiser(f):
    y, w, truth = weighted_data(f, seed=1)
    res = O.MSTEP[f](w, y, truth)
    names = synth.PARAM_NAMES[f]
    x0 = [truth[k] * 1.7 + (0.5 if k == "mu" else 0.0) for k in names]
    bounds = [(None, None) if k == "mu" else (1e-6, None) for k in names]
    opt = optimize.minimize(neg_q(f, w, y), x0, method="L-BFGS-B", bounds=bounds,
                            options=dict(ftol=1e-15, gtol=1e-12, maxiter=5000))
    for k, v in zip(names, opt.x):
        np.testing.assert_allclose(res[k], v, rtol=2e-5, err_msg=f"{f}.{k}")
    # and no better point nearby
    f0 = neg_q(f, w, y)([res[k] for k in names])
    for k in range(len(names)):
        for sgn in (-1, 1):
            th = [res[n] for n in names]
            th[k] *= 1 + sgn * 1e-4
            assert neg_q(f, w, y)(th) >= f0 - 1e-9


def test_chisq_score_equation_and_scipy_fit():
    from scipy import special as sp
    y, w, truth = weighted_data("chisq", seed=2)
    nu = O.mstep_chisq(w, y, truth)["nu"]
    c = np.sum(w * np.log(y)) / w.sum() - np.log(2.0)
    assert abs(sp.digamma(nu / 2) - c) < 1e-12
    # unit weights: the library's maximum-likelihood fit with loc 0, scale 1
    nu1 = O.mstep_chisq(np.ones_like(y), y, truth)["nu"]
    df, loc, scale = stats.chi2.fit(y, floc=0, fscale=1)
    np.testing.assert_allclose(nu1, df, rtol=1e-4)


@pytest.mark.parametrize("f", ["uniform", "pareto"])
def test_support_mstep(f):
    """The new bounds are the extremes of the rows in the current support;
    any tighter bound drops a row of positive weight (-inf objective)."""
    rng = np.random.default_rng(3)
    y = rng.uniform(0.5, 4.0, 300)
    w = rng.uniform(0.1, 1.0, 300)
    if f == "uniform":
        cur = dict(a=1.0, b=3.0)
        res = O.mstep_uniform(w, y, cur)
        inside = y[(y >= 1.0) & (y <= 3.0)]
        assert res["a"] == inside.min() and res["b"] == inside.max()
    else:
        cur = dict(xm=1.2, alpha=2.0)
        res = O.mstep_pareto(w, y, cur)
        inside = y >= 1.2
        xm = y[inside].min()
        assert res["xm"] == xm
        # alpha is the 1-D maximiser at that xm (weights outside the support are 0 here)
        ww = np.where(inside, w, 0.0)
        res = O.mstep_pareto(ww, y, cur)
        fn = lambda a: -np.sum(ww * (np.log(a) + a * np.log(xm) - (a + 1) * np.log(np.where(inside, y, 1.0))))
        opt = optimize.minimize_scalar(fn, bounds=(1e-3, 100), method="bounded", options=dict(xatol=1e-12))
        np.testing.assert_allclose(res["alpha"], opt.x, rtol=1e-6)
        # a larger xm leaves the row at the minimum outside the support
        m = model("pareto", xm=[xm * (1 + 1e-9)], alpha=[res["alpha"]])
        assert not np.isfinite(np.sum(ww[inside] * O.emission_logpdf(m, y[inside])[:, 0]))


@pytest.mark.parametrize("f", ["uniform", "pareto"])
def test_support_rows_are_the_positive_posterior_rows(f):
    ms = synth.small_models(f, 3, 1, seed=40)
    values, offsets, _ = synth.make_batch(41, ms, [60, 45], [0, 0])
    m = O.Model(f, ms[0]["pi"], ms[0]["A"], ms[0]["params"])
    assert np.all(m.A > 0) and np.all(m.pi > 0)
    for s in range(2):
        y = values[offsets[s]:offsets[s + 1]]
        g = O.forward_backward(m, y)["gamma"]
        for j in range(3):
            cur = {k: v[j] for k, v in m.params.items()}
            np.testing.assert_array_equal(g[:, j] > 0, O.support_rows(f, y, cur))


@pytest.mark.parametrize("f", FAMS)
def test_em_is_monotone(f):
    ms = synth.small_models(f, 4, 2, seed=50)
    values, offsets, mid = synth.make_batch(51, ms, [80, 33, 61, 7], [0, 1, 0, 1])
    rng = np.random.default_rng(52)
    init = [synth.perturb(rng, m) for m in ms]
    _, trace = O.fit([O.Model(f, m["pi"], m["A"], m["params"]) for m in init], values, offsets, mid, 6)
    tot = trace.sum(axis=1)
    assert np.all(np.isfinite(tot))
    assert np.all(np.diff(tot) >= -1e-8 * np.abs(tot[1:]))
