"""Pins of the oracle's emission densities and M-steps against independent
library implementations (scipy.stats densities and maximum-likelihood
fits), closed forms, score equations and the paper's worked example."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.special import digamma, polygamma

from oracle import hmm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def M(family, N=3, **params):
    return O.Model(family, np.full(N, 1.0 / N), np.full((N, N), 1.0 / N),
                   {k: np.asarray(v, np.float64) for k, v in params.items()})


# ---------------------------------------------------------------- densities
def test_emission_densities_vs_scipy():
    rng = np.random.default_rng(1)
    y = rng.normal(0, 2, 40)
    yp = rng.gamma(2.0, 1.5, 40)
    yc = rng.poisson(4.0, 40).astype(float)
    yb = rng.beta(2, 3, 40)
    cases = [
        (M("gauss", 2, mu=[0.3, -1], sigma2=[0.7, 2.5]), y,
         lambda j, yy: stats.norm.logpdf(yy, [0.3, -1][j], math.sqrt([0.7, 2.5][j]))),
        (M("poisson", 2, lam=[3.0, 7.5]), yc,
         lambda j, yy: stats.poisson.logpmf(yy, [3.0, 7.5][j])),
        (M("gamma", 2, alpha=[2.2, 0.7], beta=[1.3, 0.4]), yp,
         lambda j, yy: stats.gamma.logpdf(yy, [2.2, 0.7][j], scale=1 / [1.3, 0.4][j])),
        (M("beta", 2, a=[2.0, 0.6], b=[3.0, 1.7]), yb,
         lambda j, yy: stats.beta.logpdf(yy, [2.0, 0.6][j], [3.0, 1.7][j])),
        (M("weibull", 2, k=[1.7, 0.8], lam=[2.0, 0.9]), yp,
         lambda j, yy: stats.weibull_min.logpdf(yy, [1.7, 0.8][j], scale=[2.0, 0.9][j])),
        (M("negbin", 2, r=[2.5, 7.0], p=[0.3, 0.6]), yc,
         lambda j, yy: stats.nbinom.logpmf(yy, [2.5, 7.0][j], [0.3, 0.6][j])),
        (M("student_t", 2, mu=[0.5, -2], sigma2=[1.2, 0.3], nu=[4.0, 25.0]), y,
         lambda j, yy: stats.t.logpdf(yy, [4.0, 25.0][j], [0.5, -2][j],
                                      math.sqrt([1.2, 0.3][j]))),
        (M("vonmises", 2, mu=[0.4, -2.5], kappa=[3.0, 150.0]), y,
         lambda j, yy: stats.vonmises.logpdf(yy, [3.0, 150.0][j], loc=[0.4, -2.5][j])),
    ]
    for model, yy, ref in cases:
        lb = O.emission_logpdf(model, yy)
        for j in range(lb.shape[1]):
            r = ref(j, yy)
            if model.family == "vonmises":
                # scipy wraps y into [-pi, pi) around loc; the density is 2pi periodic
                r = stats.vonmises.logpdf(np.angle(np.exp(1j * (yy - model.params["mu"][j]))),
                                          model.params["kappa"][j])
            np.testing.assert_allclose(lb[:, j], r, rtol=1e-10, atol=1e-10,
                                       err_msg=model.family)


def test_multivariate_densities_vs_scipy():
    rng = np.random.default_rng(2)
    D, N = 3, 2
    y = rng.normal(0, 1, (25, D))
    mu = rng.normal(0, 1, (N, D))
    var = rng.uniform(0.3, 2, (N, D))
    lb = O.emission_logpdf(M("diag_gauss", N, mu=mu, var=var), y)
    G = rng.normal(0, 1, (N, D, D))
    cov = np.einsum("nij,nkj->nik", G, G) + 0.5 * np.eye(D)
    lf = O.emission_logpdf(M("full_gauss", N, mu=mu, cov=cov), y)
    for j in range(N):
        np.testing.assert_allclose(
            lb[:, j], stats.multivariate_normal.logpdf(y, mu[j], np.diag(var[j])), rtol=1e-10)
        np.testing.assert_allclose(
            lf[:, j], stats.multivariate_normal.logpdf(y, mu[j], cov[j]), rtol=1e-10)


def test_out_of_support_is_minus_inf():
    assert np.all(O.emission_logpdf(M("gamma", 1, alpha=[2.], beta=[1.]), np.array([0., -1.])) == -np.inf)
    assert np.all(O.emission_logpdf(M("poisson", 1, lam=[2.]), np.array([1.5, -1.])) == -np.inf)
    assert np.all(O.emission_logpdf(M("beta", 1, a=[2.], b=[2.]), np.array([0., 1.])) == -np.inf)


def test_golden_vonmises_wind_example():
    g = json.load(open(os.path.join(GOLDEN, "vonmises_wind_example.json")))
    y, mu = math.radians(g["y_deg"]), math.radians(g["mu_deg"])
    m = M("vonmises", 1, mu=[mu], kappa=[1.0])
    lb = O.emission_logpdf(m, np.array([y]))[0, 0]
    # log b = kappa cos(y - mu) - log(2 pi I0(kappa)) at kappa = 1
    cos_term = lb + math.log(2 * math.pi) + math.log(np.i0(1.0))
    assert round(cos_term, g["printed_decimals"]) == g["cos_term"]


# ---------------------------------------------------------------- M-steps
def fit_state(family, y, w=None, cur=None, **kw):
    w = np.ones(len(y)) if w is None else w
    return O.MSTEP[family](w, y, cur or {}, **kw)


def test_closed_forms_unit_weights():
    rng = np.random.default_rng(3)
    y = rng.normal(2, 3, 5000)
    r = fit_state("gauss", y)
    assert abs(r["mu"] - y.mean()) < 1e-12 and abs(r["sigma2"] - y.var()) < 1e-10
    c = rng.poisson(6, 5000).astype(float)
    assert abs(fit_state("poisson", c)["lam"] - c.mean()) < 1e-12
    Y = rng.normal(0, 1, (3000, 4)) * [1, 2, 3, 4]
    r = fit_state("diag_gauss", Y)
    np.testing.assert_allclose(r["mu"], Y.mean(0), atol=1e-12)
    np.testing.assert_allclose(r["var"], Y.var(0), rtol=1e-12)
    r = fit_state("full_gauss", Y)
    np.testing.assert_allclose(r["cov"], np.cov(Y.T, bias=True) + 1e-6 * np.eye(4), rtol=1e-10)


def test_closed_forms_hard_weights_are_cluster_mles():
    rng = np.random.default_rng(4)
    y = rng.normal(0, 1, 1000)
    w = (rng.random(1000) < 0.3).astype(float)
    r = fit_state("gauss", y, w)
    sub = y[w == 1]
    assert abs(r["mu"] - sub.mean()) < 1e-12 and abs(r["sigma2"] - sub.var()) < 1e-12
    ang = rng.vonmises(1.0, 4.0, 1000)
    r = fit_state("vonmises", ang, w)
    s = ang[w == 1]
    assert abs(r["mu"] - math.atan2(np.sin(s).sum(), np.cos(s).sum())) < 1e-12


def test_gamma_newton_vs_scipy_fit():
    rng = np.random.default_rng(5)
    y = rng.gamma(3.7, 1 / 2.2, 20000)
    r = fit_state("gamma", y)
    a, loc, scale = stats.gamma.fit(y, floc=0)
    assert abs(r["alpha"] - a) < 1e-4 * a and abs(1 / r["beta"] - scale) < 1e-4 * scale
    c = np.log(y.mean()) - np.log(y).mean()
    assert abs(np.log(r["alpha"]) - digamma(r["alpha"]) - c) < 1e-12   # Eq. 7 score = 0
    assert 1 <= r["_iters"] <= 8


def test_beta_newton_vs_scipy_fit():
    rng = np.random.default_rng(6)
    y = rng.beta(2.5, 4.0, 20000)
    r = fit_state("beta", y)
    a, b, _, _ = stats.beta.fit(y, floc=0, fscale=1)
    assert abs(r["a"] - a) < 1e-4 * a and abs(r["b"] - b) < 1e-4 * b
    # Eq. 9-10 at the solution
    assert abs(digamma(r["a"]) - digamma(r["a"] + r["b"]) - np.log(y).mean()) < 1e-11
    assert abs(digamma(r["b"]) - digamma(r["a"] + r["b"]) - np.log1p(-y).mean()) < 1e-11


def test_weibull_newton_vs_scipy_fit():
    rng = np.random.default_rng(7)
    y = 1.8 * rng.weibull(2.3, 20000)
    r = fit_state("weibull", y)
    k, _, lam = stats.weibull_min.fit(y, floc=0)
    assert abs(r["k"] - k) < 1e-4 * k and abs(r["lam"] - lam) < 1e-4 * lam


def test_vonmises_kappa_vs_scipy_fit():
    rng = np.random.default_rng(8)
    y = rng.vonmises(-2.0, 6.5, 20000)
    r = fit_state("vonmises", y)
    kap, loc, _ = stats.vonmises.fit(y, fscale=1)
    assert abs(r["kappa"] - kap) < 1e-4 * kap
    assert abs(np.angle(np.exp(1j * (r["mu"] - loc)))) < 1e-4
    R = np.hypot(np.cos(y).sum(), np.sin(y).sum()) / len(y)
    assert abs(O.bessel_ratio(r["kappa"]) - R) < 1e-12                # Eq. 12 fixed point


def _weighted_ll(family, theta, w, y):
    if family == "negbin":
        r = theta
        p = r / (r + np.sum(w * y) / w.sum())
        return np.sum(w * stats.nbinom.logpmf(y, r, p))
    raise ValueError


def test_negbin_profile_score_and_recovery():
    rng = np.random.default_rng(9)
    y = rng.negative_binomial(4.0, 0.35, 40000).astype(float)
    w = rng.uniform(0.2, 1.0, len(y))
    r = fit_state("negbin", y, w)
    # the profiled weighted log-likelihood (scipy pmf) is maximal at r
    f0 = _weighted_ll("negbin", r["r"], w, y)
    for h in (1e-3, -1e-3):
        assert _weighted_ll("negbin", r["r"] * (1 + h), w, y) < f0
    ybar = np.sum(w * y) / w.sum()
    assert abs(r["p"] - r["r"] / (r["r"] + ybar)) < 1e-14
    assert abs(r["r"] - 4.0) < 0.25
    under = fit_state("negbin", rng.poisson(3.0, 5000).astype(float) * 0 + 2.0)
    assert under["r"] == O.NEGBIN_RMAX


def test_student_t_ecm_fixed_point_is_mle():
    """The ECM reading (score of Eq. 18 plus the E[log U] constant) has the
    observed-data MLE as its fixed point: iterate it from a start and compare
    with scipy's maximum-likelihood t fit.  The literal Eq. 18 does not."""
    rng = np.random.default_rng(10)
    y = 0.7 + 1.3 * rng.standard_t(5.0, 20000)
    cur = dict(mu=0.0, sigma2=1.0, nu=10.0)
    for _ in range(400):
        cur = {k: v for k, v in fit_state("student_t", y, cur=cur).items() if k != "_iters"}
    df, loc, scale = stats.t.fit(y)
    assert abs(cur["nu"] - df) < 2e-3 * df
    assert abs(cur["mu"] - loc) < 1e-3
    assert abs(math.sqrt(cur["sigma2"]) - scale) < 1e-3 * scale
    lit = dict(mu=0.0, sigma2=1.0, nu=10.0)
    for _ in range(200):
        lit = {k: v for k, v in fit_state("student_t", y, cur=lit, nu_mode="paper_literal").items()
               if k != "_iters"}
    assert lit["nu"] > 2 * df      # biased upward, as the reading says


def test_student_t_cm1_closed_form():
    rng = np.random.default_rng(12)
    y = rng.standard_t(4.0, 300)
    w = rng.uniform(0, 1, 300)
    cur = dict(mu=0.2, sigma2=1.5, nu=6.0)
    r = fit_state("student_t", y, w, cur=cur)
    u = (cur["nu"] + 1) / (cur["nu"] + (y - cur["mu"]) ** 2 / cur["sigma2"])   # Eq. 14
    mu = np.sum(w * u * y) / np.sum(w * u)                                   # Eq. 15
    assert abs(r["mu"] - mu) < 1e-12
    assert abs(r["sigma2"] - np.sum(w * u * (y - mu) ** 2) / w.sum()) < 1e-12  # Eq. 16
    # CM-step 2: the nu equation is zero at the returned nu
    Nj = w.sum()
    C = np.sum(w * (np.log(u) - u)) + Nj * (digamma(3.5) - np.log(3.5))
    g = 0.5 * Nj * (np.log(r["nu"] / 2) + 1 - digamma(r["nu"] / 2)) + 0.5 * C
    assert abs(g) < 1e-6 * Nj or r["nu"] in (O.NU_MIN, O.NU_MAX)


@pytest.mark.parametrize("family,gen", [
    ("gamma", lambda r, n: r.gamma(2.0, 1.0, n)),
    ("beta", lambda r, n: r.beta(2.0, 5.0, n)),
    ("weibull", lambda r, n: 2 * r.weibull(1.5, n)),
    ("vonmises", lambda r, n: r.vonmises(0.5, 3.0, n)),
])
def test_weighted_stationarity_fractional_weights(family, gen):
    """With fractional weights the returned parameters make the gradient
    of sum_t w_t log b(y_t | theta) vanish (numerical derivative of the
    scipy density, independent of the oracle's own log-density)."""
    rng = np.random.default_rng(13)
    y = gen(rng, 5000)
    w = rng.uniform(0.05, 1.0, 5000)
    r = fit_state(family, y, w)
    if family == "gamma":
        f = lambda a, b: np.sum(w * stats.gamma.logpdf(y, a, scale=1 / b))
        th = [r["alpha"], r["beta"]]
    elif family == "beta":
        f = lambda a, b: np.sum(w * stats.beta.logpdf(y, a, b))
        th = [r["a"], r["b"]]
    elif family == "weibull":
        f = lambda k, l: np.sum(w * stats.weibull_min.logpdf(y, k, scale=l))
        th = [r["k"], r["lam"]]
    else:
        f = lambda m, k: np.sum(w * stats.vonmises.logpdf(np.angle(np.exp(1j * (y - m))), k))
        th = [r["mu"], r["kappa"]]
    for i in range(2):
        h = 1e-5 * max(1.0, abs(th[i]))
        tp, tm = list(th), list(th)
        tp[i] += h
        tm[i] -= h
        grad = (f(*tp) - f(*tm)) / (2 * h)
        assert abs(grad) < 1e-4 * w.sum(), (family, i, grad)


def test_collapse_guard_keeps_parameters():
    m = M("gauss", 2, mu=[0.0, 5.0], sigma2=[1.0, 2.0])
    y = np.linspace(-1, 1, 50)
    W = np.zeros((50, 2))
    W[:, 0] = 1.0
    W[:, 1] = 1e-12
    new, _ = O.mstep_emission(m, W, y)
    assert new.params["mu"][1] == 5.0 and new.params["sigma2"][1] == 2.0
    assert abs(new.params["mu"][0] - y.mean()) < 1e-14


def test_transition_update_matches_expected_counts():
    # with a hard (known) path the expected counts are plain transition counts
    q = np.array([0, 0, 1, 1, 1, 0, 2, 2, 0])
    N = 3
    xi = np.zeros((N, N))
    for a, b in zip(q[:-1], q[1:]):
        xi[a, b] += 1
    g1 = np.eye(N)[q[0]]
    m = M("gauss", N, mu=[0, 0, 0], sigma2=[1, 1, 1])
    pi, A = O.mstep_transitions(m, xi, g1, 1)
    np.testing.assert_allclose(A, xi / xi.sum(1, keepdims=True))
    np.testing.assert_allclose(pi, g1)


def test_special_function_values():
    eg = 0.5772156649015329
    assert abs(O.digamma(1.0) + eg) < 1e-14
    assert abs(O.digamma(0.5) + eg + 2 * math.log(2)) < 1e-14
    assert abs(O.trigamma(1.0) - math.pi ** 2 / 6) < 1e-13
    assert abs(O.trigamma(0.5) - math.pi ** 2 / 2) < 1e-13
    # A(kappa) small-argument series kappa/2 - kappa^3/16 and the large-kappa
    # asymptote 1 - 1/(2 kappa)
    assert abs(O.bessel_ratio(1e-3) - (5e-4 - 1e-9 / 16)) < 1e-15
    assert abs(O.bessel_ratio(1e4) - (1 - 1 / 2e4 - 1 / (8e8))) < 1e-11


def test_undefined_update_keeps_parameters():
    """Reading of the Sec. 4.4 guard: a state whose weighted data make the
    update undefined (zero variance, zero rate) keeps its parameters, while
    the other states update."""
    y = np.array([0.0, 1.0, 2.0, 3.0, 4.0])
    W = np.zeros((5, 2))
    W[2, 0] = 1.0                      # state 0: one observation -> variance 0
    W[:, 1] = 1.0                      # state 1: all observations
    m = O.Model("gauss", np.array([0.5, 0.5]), np.full((2, 2), 0.5),
                {"mu": np.array([7.0, 8.0]), "sigma2": np.array([3.0, 4.0])})
    new, _ = O.mstep_emission(m, W, y)
    assert new.params["mu"][0] == 7.0 and new.params["sigma2"][0] == 3.0
    assert new.params["mu"][1] == 2.0 and abs(new.params["sigma2"][1] - 2.0) < 1e-12
    yp = np.array([0.0, 0.0, 3.0])
    Wp = np.array([[1.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    mp = O.Model("poisson", np.array([0.5, 0.5]), np.full((2, 2), 0.5), {"lam": np.array([2.5, 1.0])})
    newp, _ = O.mstep_emission(mp, Wp, yp)
    assert newp.params["lam"][0] == 2.5 and newp.params["lam"][1] == 3.0
    assert O.valid_update("full_gauss", {"mu": np.zeros(2), "cov": np.eye(2)})
    assert not O.valid_update("full_gauss", {"mu": np.zeros(2), "cov": np.array([[1.0, 2.0], [2.0, 1.0]])})


def test_discrete_emission_and_mstep():
    """Categorical family (Sec. 4, 'Discrete'): log b_j(k) = log p_jk, symbols
    outside 0..K-1 (or not integers) have density 0; the M-step is the
    weighted symbol frequency -- with hard 0/1 weights, each cluster's
    empirical frequencies; with N = 1, the overall frequencies."""
    p = np.array([[0.5, 0.25, 0.25], [0.1, 0.1, 0.8]])
    m = O.Model("discrete", np.array([0.5, 0.5]), np.full((2, 2), 0.5), {"p": p.copy()})
    y = np.array([0.0, 2.0, 1.0, 3.0, 0.5, -1.0])
    lb = O.emission_logpdf(m, y)
    np.testing.assert_allclose(lb[:3], np.log(p[:, [0, 2, 1]]).T)
    assert np.all(np.isneginf(lb[3:]))
    rng = np.random.default_rng(0)
    ys = rng.integers(0, 3, 500).astype(float)
    lab = rng.integers(0, 2, 500)
    W = np.stack([(lab == 0), (lab == 1)], axis=1).astype(float)
    new, _ = O.mstep_emission(m, W, ys)
    for j in range(2):
        freq = np.bincount(ys[lab == j].astype(int), minlength=3) / (lab == j).sum()
        np.testing.assert_allclose(new.params["p"][j], freq, rtol=1e-12)
    m1 = O.Model("discrete", np.array([1.0]), np.ones((1, 1)), {"p": np.array([[0.2, 0.3, 0.5]])})
    new1, _ = O.mstep_emission(m1, np.ones((500, 1)), ys)
    np.testing.assert_allclose(new1.params["p"][0], np.bincount(ys.astype(int), minlength=3) / 500, rtol=1e-12)


def test_discrete_recursions_brute_force():
    """Forward-backward and Viterbi with categorical emissions against the
    enumeration of all N^T paths (N = 3, T = 6)."""
    rng = np.random.default_rng(4)
    N, K, T = 3, 4, 6
    m = O.Model("discrete", rng.dirichlet(np.ones(N)), rng.dirichlet(np.ones(N), size=N),
                {"p": rng.dirichlet(np.ones(K), size=N)})
    y = rng.integers(0, K, T).astype(float)
    logb = O.emission_logpdf(m, y)
    bf = O.brute_force(np.log(m.pi), np.log(m.A), logb)
    fb = O.forward_backward(m, y)
    assert abs(fb["logL"] - bf["logL"]) < 1e-12
    np.testing.assert_allclose(fb["gamma"], bf["gamma"], atol=1e-12)
    q, sc = O.viterbi(m, y)
    np.testing.assert_array_equal(q, bf["map_path"])
    assert abs(sc - bf["map_score"]) < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_transition_and_initial_update_vs_brute_force(N):
    """The transition / initial M-step of one Baum-Welch iteration against
    expected counts by enumeration of every state path: a_ij = sum over
    sequences of E[#(i -> j)] / sum over sequences of sum_{t < T} P(q_t = i),
    pi_j = mean over sequences of P(q_1 = j).  The batch mixes lengths 1..6
    so that a length-1 sequence adds to pi but not to A."""
    rng = np.random.default_rng(40 + N)
    pi = rng.dirichlet(np.ones(N))
    A = rng.dirichlet(np.ones(N), size=N)
    m = M("gauss", N, mu=list(np.linspace(-1, 1, N)), sigma2=list(rng.uniform(0.5, 2, N)))
    m.pi, m.A = pi, A
    lengths = [6, 1, 4, 5, 2]
    seqs = [rng.normal(0, 1.5, T) for T in lengths]
    values = np.concatenate(seqs)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    mid = np.zeros(len(lengths), np.int32)
    new, _ = O.em_iteration([m], values, offsets, mid)
    xi = np.zeros((N, N))
    den = np.zeros(N)
    g1 = np.zeros(N)
    for y in seqs:
        logb = O.emission_logpdf(m, y)
        bf = O.brute_force(np.log(pi), np.log(A), logb)
        xi += bf["xi_sum"]
        den += bf["gamma"][:-1].sum(axis=0)
        g1 += bf["gamma"][0]
    np.testing.assert_allclose(new[0].A, xi / den[:, None], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(new[0].pi, g1 / len(seqs), rtol=1e-11, atol=1e-13)


def test_unresolvable_variance_keeps_parameters():
    """Reading 14: a variance that vanishes relative to the weighted mean
    square deviation from the current location (here: one observation
    carrying all the weight) is an undefined update; the state keeps its
    parameters."""
    y = np.array([3.0, -1.0, 7.0])
    W = np.array([[1.0, 0.5], [0.0, 0.5], [0.0, 1.0]])
    for fam, extra in (("gauss", {}), ("student_t", {"nu": [5.0, 5.0]}), ("lognormal", {})):
        yy = np.abs(y) if fam == "lognormal" else y
        m = M(fam, 2, mu=[0.5, 0.2], sigma2=[2.0, 3.0], **extra)
        new, _ = O.mstep_emission(m, W, yy)
        assert new.params["mu"][0] == 0.5 and new.params["sigma2"][0] == 2.0, fam
        assert new.params["sigma2"][1] != 3.0, fam   # the other state is updated
