"""Pins of the oracle's k-means++ / Lloyd reading (Sec. 4.5 initialisation):
the seeding rule by hand on a tiny example, the converged state as a fixed
point (nearest-centre labels, centres at the cluster means), agreement
with scipy's Lloyd iterations from the same seeds, and recovery of
well-separated clusters."""
import numpy as np
import pytest
from scipy.cluster.vq import kmeans2

from oracle import hmm_oracle as O


def test_seeding_rule_worked_example():
    # points 0, 1, 10 (1-D); u0 = 0.5 picks index 1 (x = 1); D2 = (1, 0, 81),
    # total 82: u1 = 0.5 -> target 41, first running sum above it is index 2
    # (1, 1, 82); u1 = 0.005 -> target 0.41 -> index 0.
    X = np.array([0.0, 1.0, 10.0])
    C, _, _ = O.kmeanspp(X, [0.5, 0.5], max_iter=0)
    np.testing.assert_array_equal(C[:, 0], [1.0, 10.0])
    C, _, _ = O.kmeanspp(X, [0.5, 0.005], max_iter=0)
    np.testing.assert_array_equal(C[:, 0], [1.0, 0.0])
    # all points equal: the total is 0 and the index is floor(u T)
    C, _, _ = O.kmeanspp(np.ones(4), [0.1, 0.8], max_iter=0)
    np.testing.assert_array_equal(C[:, 0], [1.0, 1.0])


@pytest.mark.parametrize("K,F", [(2, 1), (3, 2), (8, 3)])
def test_lloyd_fixed_point_and_scipy(K, F):
    rng = np.random.default_rng(K * 10 + F)
    X = rng.normal(0, 1, (3000, F)) + rng.integers(0, K, 3000)[:, None] * 3.0
    X = X.astype(np.float32).astype(np.float64)
    u = rng.random(K)
    C, lab, passes = O.kmeanspp(X, u, max_iter=200)
    assert passes < 200
    d = np.sum((X[:, None, :] - C[None]) ** 2, axis=2)
    np.testing.assert_array_equal(lab, np.argmin(d, axis=1))
    for j in range(K):
        if np.any(lab == j):
            np.testing.assert_allclose(C[j], X[lab == j].mean(axis=0), rtol=1e-12, atol=1e-12)
    # the same Lloyd iterations in scipy from the same seeds
    C0, _, _ = O.kmeanspp(X, u, max_iter=0)
    Cs, ls = kmeans2(X, C0.copy(), iter=passes + 5, minit="matrix", missing="raise")
    np.testing.assert_allclose(Cs, C, rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(ls, lab)


def test_well_separated_clusters_recovered():
    rng = np.random.default_rng(3)
    means = np.array([-10.0, 0.0, 10.0])
    z = rng.integers(0, 3, 5000)
    X = means[z] + rng.normal(0, 1, 5000)
    C, lab, _ = O.kmeanspp(X, rng.random(3))
    np.testing.assert_allclose(np.sort(C[:, 0]), means, atol=0.1)
    order = np.argsort(C[:, 0])
    rank = np.empty(3, int)
    rank[order] = np.arange(3)
    assert np.mean(rank[lab] == z) > 0.999
