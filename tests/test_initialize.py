"""k-means++ starting parameters (host, input preparation): seeded,
deterministic, row-stochastic, and the cluster moments of separated data."""
import numpy as np

from paper_2605_29208_gb300 import initialize, synth


def test_kmeanspp_separated_clusters():
    rng = np.random.default_rng(0)
    y = np.concatenate([rng.normal(-5, 1, 400), rng.normal(5, 1, 600)])
    rng.shuffle(y)
    m = initialize.kmeanspp_init("gauss", 2, y, np.array([0, len(y)]), seed=1)
    np.testing.assert_allclose(m["params"]["mu"], [-5, 5], atol=0.2)
    np.testing.assert_allclose(m["params"]["sigma2"], [1, 1], atol=0.25)
    np.testing.assert_allclose(m["A"].sum(axis=1), 1.0)
    np.testing.assert_allclose(m["pi"], 0.5)


def test_kmeanspp_deterministic_and_transitions():
    truth, values, offsets, mid = synth.tiny_gauss()
    a = initialize.kmeanspp_init("gauss", 2, values, offsets, seed=3)
    b = initialize.kmeanspp_init("gauss", 2, values, offsets, seed=3)
    for k in a["params"]:
        np.testing.assert_array_equal(a["params"][k], b["params"][k])
    np.testing.assert_array_equal(a["A"], b["A"])
    # the sticky chain (a_ii = 0.9) shows in the label transitions
    assert a["A"][0, 0] > 0.6 and a["A"][1, 1] > 0.6
    assert a["params"]["mu"][0] < 0 < a["params"]["mu"][1]


def test_kmeanspp_families():
    rng = np.random.default_rng(2)
    for fam, D in (("poisson", 1), ("gamma", 1), ("vonmises", 1), ("diag_gauss", 3), ("full_gauss", 3)):
        models = synth.small_models(fam, 3, 1, seed=5, D=D)
        values, offsets, _ = synth.make_batch(6, models, [300, 200], [0, 0])
        if D > 1:
            values = values.reshape(-1, D)
        m = initialize.kmeanspp_init(fam, 3, values, offsets, seed=1)
        assert m["family"] == fam
        for k, v in m["params"].items():
            assert np.all(np.isfinite(v)), (fam, k)
        np.testing.assert_allclose(m["A"].sum(axis=1), 1.0)
