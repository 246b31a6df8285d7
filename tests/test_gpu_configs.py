"""The small end-to-end configuration: a 2-state univariate Gaussian HMM
(means -1, +1, sd 1, a_ii = 0.9), one sequence of T = 1000, 20 Baum-Welch
iterations from the k-means++ start, then Viterbi -- on the CUDA path
against the FP64 oracle run from the same start."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import initialize, synth
from parity import assert_params_close, check_fit_iterations, check_viterbi_fp64

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


def test_tiny_gauss_fit_and_decode(H):
    truth, values, offsets, mid = synth.tiny_gauss()
    ctx = H.Context(0)
    init = initialize.kmeanspp_init("gauss", 2, values, offsets, seed=0, ctx=ctx)
    model = H.Model(ctx, [init])
    batch = H.Batch(values, offsets, mid)
    trace, (ref_models, ref_trace) = check_fit_iterations(H, ctx, model, batch, values, offsets, mid, 20)
    np.testing.assert_allclose(trace[:, 0], ref_trace.sum(axis=1), rtol=1e-5)
    got = model.get()[0]
    ref = ref_models[0]
    assert_params_close([got], [ref], rtol=1e-4)
    # the fit lands near the generating parameters
    np.testing.assert_allclose(np.sort(got["params"]["mu"]), [-1, 1], atol=0.25)
    # EM never decreases the likelihood
    assert np.all(np.diff(trace[:, 0]) >= -1e-6 * abs(trace[0, 0]))
    path, score = H.viterbi(ctx, model, batch)
    path = path.cpu().numpy()
    score = float(score.cpu().numpy()[0])
    check_viterbi_fp64(path, score, ref, values, where="tiny")
