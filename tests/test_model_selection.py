"""Model-selection criteria (AIC, BIC, AICc; the paper names them without
formulas): the oracle's free-parameter count against counts done by hand,
the criteria against their textbook values, and the library's host-side
hmm_information_criteria against the oracle for every family (no GPU)."""
import math

import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth


def om(d):
    return O.Model(d["family"], d["pi"], d["A"], d["params"])


@pytest.mark.parametrize("family,N,D,k", [
    ("gauss", 2, 1, 1 + 2 + 2 * 2),            # pi 1, A 2, (mu, sigma2) x 2
    ("discrete", 3, 4, 2 + 6 + 3 * 3),         # pi 2, A 6, 3 free symbol probabilities x 3
    ("full_gauss", 2, 3, 1 + 2 + 2 * (3 + 6)),  # mean 3 + 6 covariance entries per state
    ("diag_gauss", 4, 2, 3 + 12 + 4 * 4),
    ("student_t", 3, 1, 2 + 6 + 3 * 3),
    ("exponential", 5, 1, 4 + 20 + 5),
])
def test_free_parameters_by_hand(family, N, D, k):
    m = synth.small_models(family, N, 1, seed=3, D=D)[0]
    assert O.free_parameter_count(om(m)) == k


def test_textbook_values():
    m = om(synth.small_models("gauss", 2, 1, seed=1)[0])     # k = 7
    r = O.information_criteria(m, -100.0, 50)
    assert r["aic"] == pytest.approx(2 * 7 + 200.0)
    assert r["bic"] == pytest.approx(7 * math.log(50) + 200.0)
    assert r["aicc"] == pytest.approx(214.0 + 2 * 7 * 8 / (50 - 8))
    # BIC - AIC = k (ln n - 2); AICc -> AIC as n grows; AICc undefined for n <= k + 1
    assert r["bic"] - r["aic"] == pytest.approx(7 * (math.log(50) - 2))
    assert O.information_criteria(m, -100.0, 10 ** 9)["aicc"] == pytest.approx(r["aic"], rel=1e-6)
    assert O.information_criteria(m, -100.0, 8)["aicc"] == math.inf


FAMS = ["gauss", "poisson", "gamma", "beta", "weibull", "negbin", "student_t", "vonmises",
        "lognormal", "exponential", "rayleigh", "uniform", "chisq", "pareto"]


@pytest.mark.parametrize("family", FAMS + ["discrete", "diag_gauss", "full_gauss"])
def test_library_matches_oracle(family):
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import _lib
    try:
        _lib.load()
    except (ImportError, OSError) as e:
        pytest.skip(f"library not built: {e}")
    D = 3 if family in ("discrete", "diag_gauss", "full_gauss") else 1
    for N in (1, 2, 7):
        m = om(synth.small_models(family, N, 1, seed=5, D=D)[0])
        for ll, n in ((-1234.5, 10000), (17.0, 5), (0.0, 1)):
            ref = O.information_criteria(m, ll, n)
            got = H.information_criteria(family, N, ll, n, dim=D)
            assert got["k"] == ref["k"]
            for key in ("aic", "bic", "aicc"):
                assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-12), (family, N, key)


def test_library_rejects_bad_arguments():
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import HmmError, _lib
    try:
        _lib.load()
    except (ImportError, OSError) as e:
        pytest.skip(f"library not built: {e}")
    with pytest.raises(HmmError):
        H.information_criteria("gauss", 0, 0.0, 10)
    with pytest.raises(HmmError):
        H.information_criteria("gauss", 2, 0.0, 0)


def test_restart_batch_layout():
    """The restart batch repeats the sequences once per model, in order."""
    from paper_2605_29208_gb300.restarts import _replicate
    values = np.arange(7, dtype=np.float64)
    offsets = np.array([0, 3, 3, 7])
    vals, offs, mid = _replicate(values, offsets, 3)
    np.testing.assert_array_equal(vals, np.tile(values, 3))
    np.testing.assert_array_equal(offs, [0, 3, 3, 7, 10, 10, 14, 17, 17, 21])
    np.testing.assert_array_equal(mid, [0, 0, 0, 1, 1, 1, 2, 2, 2])
