"""The time-parallel forward-backward (HMM_OPT_TIME_PARALLEL: chunk transfer
matrices, boundary vectors, chunks recomputed in parallel) against the FP64
oracle and against the sequential recursion, with the float32 path's
tolerances: per-sequence logL 1e-5 relative, gamma 1e-4 absolute."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


def om(d):
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(),
                   {k: np.array(v, copy=True) for k, v in d["params"].items()})


def ctx_with(H, mode):
    from paper_2605_29208_gb300 import _lib
    c = H.Context(0)
    c.set_option(_lib.OPT_TIME_PARALLEL, mode)
    return c


@pytest.mark.parametrize("family,N,D", [("gauss", 2, 1), ("discrete", 3, 3), ("gamma", 8, 1), ("poisson", 16, 1),
                                        ("gauss", 32, 1), ("diag_gauss", 5, 2)])
def test_time_parallel_parity(H, family, N, D):
    lengths = [1, 2, 0, 127, 128, 129, 300, 1000, 2600]
    models = synth.small_models(family, N, 2, seed=1800 + N, D=D)
    values, offsets, mid = synth.make_batch(1801 + N, models, lengths, np.arange(len(lengths)) % 2)
    if D > 1 and family != "discrete":
        values = values.reshape(-1, D)
    ctx = ctx_with(H, 1)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid, dim=D if family not in ("discrete",) else 1)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    ll, gamma = ll.cpu().numpy(), gamma.cpu().numpy()
    for s in range(len(lengths)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        fb = O.forward_backward(om(models[mid[s]]), np.asarray(y, np.float64))
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"])), (s, ll[s], fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL, rtol=0)


@pytest.mark.parametrize("N", [2, 16])
def test_time_parallel_matches_sequential_long(H, N):
    """One sequence of 200k steps: the time-parallel result (chosen
    automatically for a single long sequence) agrees with the sequential
    recursion, and the oracle's log-likelihood on it."""
    models = synth.small_models("gauss", N, 1, seed=1900 + N, conc=0.5)
    values, offsets, mid = synth.make_batch(1901, models, [200000], [0])
    ctx_a = ctx_with(H, 0)
    ctx_s = ctx_with(H, -1)
    model_a = H.Model(ctx_a, models)
    model_s = H.Model(ctx_s, models)
    lla, ga, _ = H.forward_backward(ctx_a, model_a, H.Batch(values, offsets, mid))
    lls, gs, _ = H.forward_backward(ctx_s, model_s, H.Batch(values, offsets, mid))
    lla, lls = float(lla.cpu()[0]), float(lls.cpu()[0])
    assert abs(lla - lls) <= LL_RTOL * abs(lls)
    assert float((ga - gs).abs().max()) <= GAMMA_ATOL
    o = om(models[0])
    alpha = O.forward_log(np.log(o.pi), np.log(o.A), O.emission_logpdf(o, values))
    ref = float(O.lse(alpha[-1], axis=0))
    assert abs(lla - ref) <= LL_RTOL * abs(ref)
