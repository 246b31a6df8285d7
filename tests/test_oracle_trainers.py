"""Pins of the oracle's MAP Baum-Welch and Viterbi-training readings (the
paper names both trainers, Sec. 5.6, without definitions): the MAP
transition update against brute-force expected counts plus the Dirichlet
pseudo-counts and its monotone posterior objective; Viterbi training
against brute-force MAP paths, hard per-cluster fits and its monotone
best-path objective."""
import numpy as np
import pytest
from scipy import stats

from oracle import hmm_oracle as O


def gauss_model(N, rng):
    return O.Model("gauss", rng.dirichlet(np.ones(N)), rng.dirichlet(np.ones(N) * 2, size=N),
                   dict(mu=np.linspace(-2, 2, N) + rng.normal(0, 0.1, N), sigma2=rng.uniform(0.5, 1.5, N)))


def sample(model, lengths, rng):
    seqs = []
    for T in lengths:
        q = [rng.choice(model.n_states, p=model.pi)]
        for _ in range(T - 1):
            q.append(rng.choice(model.n_states, p=model.A[q[-1]]))
        q = np.array(q)
        seqs.append(model.params["mu"][q] + np.sqrt(model.params["sigma2"][q]) * rng.standard_normal(T))
    return np.concatenate(seqs), np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)


def test_map_with_flat_priors_is_maximum_likelihood():
    rng = np.random.default_rng(1)
    m = gauss_model(3, rng)
    values, offsets = sample(m, [200, 150, 90], rng)
    mid = np.zeros(3, np.int32)
    a, _ = O.em_iteration([m], values, offsets, mid)
    b, _ = O.em_iteration([m], values, offsets, mid, alpha_A=1.0, alpha_pi=0.5)
    np.testing.assert_array_equal(a[0].A, b[0].A)
    np.testing.assert_array_equal(a[0].pi, b[0].pi)


@pytest.mark.parametrize("N,alpha", [(2, 3.0), (3, 1.5)])
def test_map_transitions_vs_brute_force_counts(N, alpha):
    rng = np.random.default_rng(10 + N)
    m = gauss_model(N, rng)
    lengths = [6, 1, 5, 4]
    seqs = [rng.normal(0, 1.5, T) for T in lengths]
    values = np.concatenate(seqs)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    new, _ = O.em_iteration([m], values, offsets, np.zeros(4, np.int32), alpha_A=alpha, alpha_pi=alpha + 1)
    xi, g1 = np.zeros((N, N)), np.zeros(N)
    for y in seqs:
        bf = O.brute_force(np.log(m.pi), np.log(m.A), O.emission_logpdf(m, y))
        xi += bf["xi_sum"]
        g1 += bf["gamma"][0]
    c = alpha - 1
    np.testing.assert_allclose(new[0].A, (xi + c) / (xi.sum(1, keepdims=True) + N * c), rtol=1e-11)
    np.testing.assert_allclose(new[0].pi, (g1 + alpha) / (4 + N * alpha), rtol=1e-11)


def test_map_em_increases_the_posterior():
    rng = np.random.default_rng(3)
    truth = gauss_model(3, rng)
    values, offsets = sample(truth, [300, 200, 120], rng)
    mid = np.zeros(3, np.int32)
    models = [gauss_model(3, np.random.default_rng(99))]
    obj = []
    for _ in range(10):
        new, ll = O.em_iteration(models, values, offsets, mid, alpha_A=2.5, alpha_pi=2.0)
        obj.append(ll.sum() + O.log_dirichlet_prior(models[0], 2.5, 2.0))
        models = new
    assert np.all(np.diff(obj) >= -1e-9 * abs(obj[0]))


def test_viterbi_estep_paths_and_counts_vs_brute_force():
    rng = np.random.default_rng(4)
    m = gauss_model(3, rng)
    lengths = [7, 5, 1, 6]
    seqs = [rng.normal(0, 1.5, T) for T in lengths]
    values = np.concatenate(seqs)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    res = O.viterbi_estep([m], values, offsets, np.zeros(4, np.int32))[0]
    xi, g1 = np.zeros((3, 3)), np.zeros(3)
    for y, q, sc in zip(seqs, res["path"], res["score"]):
        bf = O.brute_force(np.log(m.pi), np.log(m.A), O.emission_logpdf(m, y))
        np.testing.assert_array_equal(q, bf["map_path"])
        assert abs(sc - bf["map_score"]) < 1e-10 * abs(sc)
        for a, b in zip(q[:-1], q[1:]):
            xi[a, b] += 1
        g1[q[0]] += 1
    np.testing.assert_array_equal(res["xi_sum"], xi)
    np.testing.assert_array_equal(res["gamma1_sum"], g1)


def test_viterbi_training_mstep_is_the_per_segment_fit():
    rng = np.random.default_rng(5)
    truth = gauss_model(2, rng)
    truth.params["mu"] = np.array([-3.0, 3.0])
    values, offsets = sample(truth, [400, 300], rng)
    mid = np.zeros(2, np.int32)
    new, _ = O.viterbi_train_iteration([truth], values, offsets, mid)
    res = O.viterbi_estep([truth], values, offsets, mid)[0]
    q = np.concatenate(res["path"])
    for j in range(2):
        yj = values[q == j]
        assert abs(new[0].params["mu"][j] - yj.mean()) < 1e-12
        assert abs(new[0].params["sigma2"][j] - yj.var()) < 1e-12
    n = res["xi_sum"]
    np.testing.assert_allclose(new[0].A, n / n.sum(1, keepdims=True), rtol=1e-14)


def test_viterbi_training_objective_never_decreases():
    rng = np.random.default_rng(6)
    truth = gauss_model(3, rng)
    values, offsets = sample(truth, [250, 250, 100], rng)
    mid = np.zeros(3, np.int32)
    models = [gauss_model(3, np.random.default_rng(7))]
    obj = []
    for _ in range(12):
        models, sc = O.viterbi_train_iteration(models, values, offsets, mid)
        obj.append(sc.sum())
    assert np.all(np.diff(obj) >= -1e-9 * abs(obj[0]))
    # after convergence the paths no longer change: two more iterations keep the score
    _, s1 = O.viterbi_train_iteration(models, values, offsets, mid)
    assert abs(s1.sum() - obj[-1]) <= 1e-6 * abs(obj[-1]) or s1.sum() >= obj[-1]
