"""Random restarts in one multi-model batch and state-count selection by
BIC (paper Sec. 4.5: k-means++ starts; Sec. 5.6: AIC / BIC / AICc): every
restart in the shared batch against the FP64 oracle fitting that restart
alone, and BIC picking the generating state count on well-separated data."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth

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


def separated(N, seed):
    truth = synth.make_model("gauss", np.full(N, 1.0 / N), 0.8 * np.eye(N) + 0.2 / N,
                             mu=6.0 * np.arange(N) - 3.0 * (N - 1), sigma2=np.ones(N))
    values, offsets, _ = synth.make_batch(seed, [truth], [200] * 20, [0] * 20)
    return truth, values, offsets


def test_restarts_match_the_oracle(H):
    from paper_2605_29208_gb300 import restarts
    from paper_2605_29208_gb300.initialize import kmeanspp_init
    _, values, offsets = separated(3, 3100)
    ctx = H.Context(0)
    models, ll, crit = restarts.fit_restarts(ctx, "gauss", 3, values, offsets, n_restarts=3, n_iter=5, seed=7)
    mid = np.zeros(len(offsets) - 1, np.int32)
    for r in range(3):
        init = kmeanspp_init("gauss", 3, values, offsets, seed=7 + r, ctx=ctx)
        ref, _ = O.fit([O.Model("gauss", init["pi"], init["A"], init["params"])], values, offsets, mid, 5)
        ref_ll = O.batch_loglik(ref, values, offsets, mid).sum()
        assert abs(ll[r] - ref_ll) <= 1e-5 * abs(ref_ll)
        for k, v in ref[0].params.items():
            np.testing.assert_allclose(models[r]["params"][k], v, rtol=1e-4, atol=1e-6, err_msg=k)
        assert crit[r]["bic"] == pytest.approx(O.information_criteria(ref[0], ref_ll, int(offsets[-1]))["bic"],
                                               rel=1e-6)


def test_bic_selects_the_state_count(H):
    from paper_2605_29208_gb300 import restarts
    _, values, offsets = separated(3, 3200)
    ctx = H.Context(0)
    best, table = restarts.select_states(ctx, "gauss", [2, 3, 4], values, offsets, n_restarts=3, n_iter=15)
    assert best == 3
    assert table[3][1] > table[2][1]
