"""Pins of the oracle's independent-components family (Sec. 4.5: b_j(y) =
prod_d phi_d(y_d), each component fitted by its own scalar M-step with the
same occupancy weights) against scipy densities and fits, per-cluster
fits under hard weights, the vanishing gradient of the weighted
log-likelihood under fractional weights, brute-force path enumeration and
EM monotonicity."""
import numpy as np
import pytest
from scipy import optimize, stats

from oracle import hmm_oracle as O


def indep_model(N=2):
    rng = np.random.default_rng(1)
    params = {"d0.alpha": rng.uniform(2, 6, N), "d0.beta": rng.uniform(0.5, 2, N),
              "d1.mu": rng.uniform(-2, 2, N), "d1.kappa": rng.uniform(0.5, 5, N),
              "d2.mu": rng.normal(0, 2, N), "d2.sigma2": rng.uniform(0.5, 2, N)}
    return O.Model("indep", np.full(N, 1.0 / N), np.full((N, N), 1.0 / N), params,
                   ("gamma", "vonmises", "gauss"))


def draws(rng, T, alpha, beta, mu, kappa, m2, s2):
    return np.stack([rng.gamma(alpha, 1 / beta, T), stats.vonmises.rvs(kappa, loc=mu, size=T, random_state=rng),
                     rng.normal(m2, np.sqrt(s2), T)], axis=1)


def test_indep_density_is_the_product_of_scipy_densities():
    m = indep_model(3)
    rng = np.random.default_rng(2)
    y = np.stack([rng.gamma(3, 1, 50), rng.uniform(-np.pi, np.pi, 50), rng.normal(0, 2, 50)], axis=1)
    got = O.emission_logpdf(m, y)
    p = m.params
    ref = (stats.gamma.logpdf(y[:, :1], p["d0.alpha"], scale=1 / p["d0.beta"])
           + stats.vonmises.logpdf(y[:, 1:2], p["d1.kappa"], loc=p["d1.mu"])
           + stats.norm.logpdf(y[:, 2:3], p["d2.mu"], np.sqrt(p["d2.sigma2"])))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-10)
    # out of one component's support: density 0
    y[3, 0] = -1.0
    assert np.all(O.emission_logpdf(m, y)[3] == -np.inf)


def test_indep_mstep_with_unit_weights_matches_scipy_fits():
    rng = np.random.default_rng(3)
    y = draws(rng, 200_000, 3.0, 1.5, 0.7, 2.5, -1.0, 0.8)
    m = indep_model(1)
    new, _ = O.mstep_emission(m, np.ones((len(y), 1)), y)
    a, _, sc = stats.gamma.fit(y[:, 0], floc=0)
    k, loc, _ = stats.vonmises.fit(y[:, 1], fscale=1)
    p = new.params
    assert abs(p["d0.alpha"][0] - a) < 1e-5 * a and abs(p["d0.beta"][0] - 1 / sc) < 1e-5 / sc
    assert abs(p["d1.kappa"][0] - k) < 1e-5 * k and abs(np.angle(np.exp(1j * (p["d1.mu"][0] - loc)))) < 1e-6
    assert abs(p["d2.mu"][0] - y[:, 2].mean()) < 1e-12 and abs(p["d2.sigma2"][0] - y[:, 2].var()) < 1e-12
    # and the generating values within a few standard errors
    assert abs(p["d0.alpha"][0] - 3.0) < 0.05 and abs(p["d1.kappa"][0] - 2.5) < 0.05


def test_indep_mstep_hard_weights_are_per_cluster_fits():
    rng = np.random.default_rng(4)
    ya = draws(rng, 4000, 2.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    yb = draws(rng, 3000, 8.0, 2.0, 2.0, 6.0, 3.0, 0.5)
    y = np.concatenate([ya, yb])
    W = np.zeros((len(y), 2))
    W[:4000, 0] = 1
    W[4000:, 1] = 1
    new, _ = O.mstep_emission(indep_model(2), W, y)
    for j, part in ((0, ya), (1, yb)):
        one, _ = O.mstep_emission(indep_model(1), np.ones((len(part), 1)), part)
        for k, v in one.params.items():
            assert abs(new.params[k][j] - v[0]) <= 1e-9 * max(1, abs(v[0])), k


def test_indep_mstep_fractional_weights_zero_gradient():
    """Each component's update maximises its weighted log-likelihood: the
    numerical gradient of sum_t w_t log phi(y_t) vanishes there."""
    rng = np.random.default_rng(5)
    y = draws(rng, 3000, 4.0, 1.2, -0.5, 3.0, 1.0, 2.0)
    w = rng.uniform(0.05, 1.0, len(y))
    new, _ = O.mstep_emission(indep_model(1), w[:, None], y)
    p = {k: v[0] for k, v in new.params.items()}
    fns = {
        ("d0.alpha", "d0.beta"): lambda a, b: np.sum(w * stats.gamma.logpdf(y[:, 0], a, scale=1 / b)),
        ("d1.mu", "d1.kappa"): lambda mu, k: np.sum(w * stats.vonmises.logpdf(y[:, 1], k, loc=mu)),
        ("d2.mu", "d2.sigma2"): lambda mu, s2: np.sum(w * stats.norm.logpdf(y[:, 2], mu, np.sqrt(s2))),
    }
    for (n1, n2), f in fns.items():
        x = np.array([p[n1], p[n2]])
        g = optimize.approx_fprime(x, lambda v: f(*v), 1e-6 * np.maximum(1, np.abs(x)))
        assert np.all(np.abs(g) < 1e-3 * w.sum()), (n1, g)


def test_indep_recursions_vs_brute_force():
    m = indep_model(2)
    m.A = np.array([[0.8, 0.2], [0.3, 0.7]])
    m.pi = np.array([0.6, 0.4])
    rng = np.random.default_rng(6)
    y = draws(rng, 6, 3.0, 1.0, 0.0, 2.0, 0.0, 1.0)
    logb = O.emission_logpdf(m, y)
    fb = O.forward_backward(m, y)
    bf = O.brute_force(np.log(m.pi), np.log(m.A), logb)
    assert abs(fb["logL"] - bf["logL"]) < 1e-11 * abs(bf["logL"])
    np.testing.assert_allclose(fb["gamma"], bf["gamma"], atol=1e-12)


def test_indep_em_is_monotone_and_counts_parameters():
    rng = np.random.default_rng(7)
    truth = indep_model(2)
    truth.A = np.array([[0.9, 0.1], [0.2, 0.8]])
    seqs = []
    for _ in range(4):
        q = [0]
        for _t in range(299):
            q.append(q[-1] if rng.random() < truth.A[q[-1], q[-1]] else 1 - q[-1])
        q = np.array(q)
        p = truth.params
        seqs.append(np.stack([rng.gamma(p["d0.alpha"][q], 1 / p["d0.beta"][q]),
                              stats.vonmises.rvs(p["d1.kappa"][q], loc=p["d1.mu"][q], random_state=rng),
                              rng.normal(p["d2.mu"][q], np.sqrt(p["d2.sigma2"][q]))], axis=1))
    values = np.concatenate(seqs)
    offsets = np.array([0, 300, 600, 900, 1200])
    mid = np.zeros(4, np.int32)
    start = indep_model(2)
    models, trace = O.fit([start], values, offsets, mid, 8)
    tot = trace.sum(axis=1)
    assert np.all(np.diff(tot) >= -1e-9 * np.abs(tot).max())
    assert O.free_parameter_count(start) == 1 + 2 + 2 * 6
