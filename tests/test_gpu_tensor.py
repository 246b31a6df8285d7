"""The tensor-core recursions (HMM_OPT_TENSOR_RECURRENCE: tcgen05 GEMMs with
FP16 operands, FP32 accumulation, float64 shift) against the FP64 oracle.

The FP16 operands round every scaled vector entry and every transition
probability to 11 significant bits, so this path is held to its own stated
bounds instead of the float32 path's: per-sequence logL within 5e-5
relative, gamma within 1e-3 absolute, one EM iteration's parameters within
2e-3 relative.  Measured on GB300: logL <= 1.2e-5 relative, gamma <= 2.2e-4."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth

pytestmark = pytest.mark.gpu

TC_LL_RTOL = 5e-5
TC_GAMMA_ATOL = 1e-3
TC_PARAM_RTOL = 2e-3


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


@pytest.fixture()
def ctx(H):
    from paper_2605_29208_gb300 import _lib
    c = H.Context(0)
    c.set_option(_lib.OPT_TENSOR_RECURRENCE, 1)
    return c


def om(d):
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(),
                   {k: np.array(v, copy=True) for k, v in d["params"].items()})


def build(H, ctx, family, N, D, conc, lengths, n_models, seed):
    models = synth.small_models(family, N, n_models, seed=seed, conc=conc, D=D)
    mid = np.arange(len(lengths)) % n_models
    values, offsets, mid = synth.make_batch(seed + 1, models, lengths, mid)
    if D > 1:
        values = values.reshape(-1, D)
    return models, values, offsets, mid, H.Model(ctx, models), H.Batch(values, offsets, mid, dim=D)


# more than 128 sequences of one model: several tiles, ragged lengths, empty ones
MANY = [1 + (s * 7) % 23 for s in range(300)] + [0, 130, 257]


@pytest.mark.parametrize("family,N,D,conc,lengths,n_models", [
    ("diag_gauss", 64, 4, 1.0, [1, 2, 50, 130, 0, 7], 1),
    ("gauss", 100, 1, 1.0, MANY, 2),
    ("gamma", 200, 1, 1.0, [33, 90, 5, 1], 2),
    ("diag_gauss", 512, 8, 0.1, [1, 40, 97, 150], 1),
])
def test_tensor_forward_backward(H, ctx, family, N, D, conc, lengths, n_models):
    models, values, offsets, mid, model, batch = build(H, ctx, family, N, D, conc, lengths, n_models, 1000 + N)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    assert ctx.status() == 0
    ll = ll.cpu().numpy()
    gamma = gamma.cpu().numpy()
    for s in range(len(lengths)):
        y = np.asarray(values[offsets[s]:offsets[s + 1]], np.float64)
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        fb = O.forward_backward(om(models[mid[s]]), y)
        assert abs(ll[s] - fb["logL"]) <= TC_LL_RTOL * max(1.0, abs(fb["logL"])), (s, ll[s], fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=TC_GAMMA_ATOL, rtol=0)


@pytest.mark.parametrize("family,N,D", [("gauss", 64, 1), ("diag_gauss", 256, 3)])
def test_tensor_em_iteration(H, ctx, family, N, D):
    truth = synth.small_models(family, N, 1, seed=1100 + N, D=D)
    lengths = [400, 250, 1, 333, 128]
    values, offsets, mid = synth.make_batch(1101, truth, lengths, np.zeros(len(lengths), np.int32))
    if D > 1:
        values = values.reshape(-1, D)
    rng = np.random.default_rng(9)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid, dim=D)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in init], np.asarray(values, np.float64), offsets, mid)
    for g, r in zip(model.get(), ref):
        np.testing.assert_allclose(g["pi"], r.pi, rtol=TC_PARAM_RTOL, atol=1e-4)
        np.testing.assert_allclose(g["A"], r.A, rtol=TC_PARAM_RTOL, atol=1e-4)
        for k, v in r.params.items():
            np.testing.assert_allclose(g["params"][k], v, rtol=TC_PARAM_RTOL, atol=1e-5, err_msg=k)


def test_tensor_matches_float32_path(H, ctx):
    """Both recursions on a larger batch (N = 512, 260 sequences, Dirichlet(0.1)
    rows): the tensor path stays within its bounds of the float32 path."""
    from paper_2605_29208_gb300 import _lib
    models, values, offsets, mid, model, batch = build(H, ctx, "diag_gauss", 512, 16, 0.1, [64] * 260, 1, 1200)
    ll1, g1, _ = H.forward_backward(ctx, model, batch)
    ctx.set_option(_lib.OPT_TENSOR_RECURRENCE, 0)
    ll0, g0, _ = H.forward_backward(ctx, model, batch)
    ll0, ll1 = ll0.cpu().numpy(), ll1.cpu().numpy()
    assert np.all(np.abs(ll1 - ll0) <= TC_LL_RTOL * np.maximum(1.0, np.abs(ll0)))
    assert float((g1 - g0).abs().max()) <= TC_GAMMA_ATOL


@pytest.mark.parametrize("N", [128, 300])
def test_tensor_xi_statistics(H, ctx, N):
    """E-step statistics with the tensor-core recursions and the TF32 xi GEMM
    (K = time, chunk-ordered layout) against sums of the oracle's posteriors."""
    models = synth.small_models("gauss", N, 2, seed=1300 + N)
    lengths = [50, 3, 0, 200, 120, 1, 77, 40]
    values, offsets, mid = synth.make_batch(1301, models, lengths, np.arange(len(lengths)) % 2)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    got = stats.get()
    off = 0
    for m, md in enumerate(models):
        o = om(md)
        g1, xi, ll, W = np.zeros(N), np.zeros((N, N)), 0.0, np.zeros(N)
        idx = [s for s in range(len(lengths)) if mid[s] == m]
        for s in idx:
            y = np.asarray(values[offsets[s]:offsets[s + 1]], np.float64)
            if len(y) == 0:
                continue
            fb = O.forward_backward(o, y)
            ll += fb["logL"]
            g1 += fb["gamma"][0]
            xi += fb["xi_sum"]
            W += fb["gamma"].sum(0)
        rec = got[off:off + 2 + N + N * N + 3 * N]
        off += 2 + N + N * N + 3 * N
        assert rec[0] == len(idx)
        assert abs(rec[1] - ll) <= TC_LL_RTOL * abs(ll)
        np.testing.assert_allclose(rec[2:2 + N], g1, atol=TC_GAMMA_ATOL * len(idx))
        np.testing.assert_allclose(rec[2 + N:2 + N + N * N].reshape(N, N), xi, rtol=5e-3, atol=5e-3)
        np.testing.assert_allclose(rec[2 + N + N * N::3], W, rtol=2e-3, atol=2e-3)


# TF32 operands (HMM_OPT_TENSOR_RECURRENCE = 2, padded N <= 256): the same
# 10 significant bits as FP16 with float32's exponent range, held to the same
# stated bounds.

@pytest.fixture()
def ctx32(H):
    from paper_2605_29208_gb300 import _lib
    c = H.Context(0)
    c.set_option(_lib.OPT_TENSOR_RECURRENCE, 2)
    return c


@pytest.mark.parametrize("family,N,D,conc,lengths,n_models", [
    ("diag_gauss", 64, 4, 1.0, [1, 2, 50, 130, 0, 7], 1),
    ("gauss", 100, 1, 1.0, MANY, 2),
    ("gamma", 200, 1, 1.0, [33, 90, 5, 1], 2),
    ("diag_gauss", 256, 8, 0.1, [1, 40, 97, 150], 1),
])
def test_tf32_forward_backward(H, ctx32, family, N, D, conc, lengths, n_models):
    test_tensor_forward_backward(H, ctx32, family, N, D, conc, lengths, n_models)


def test_tf32_em_iteration(H, ctx32):
    test_tensor_em_iteration(H, ctx32, "gauss", 64, 1)


def test_tf32_xi_statistics(H, ctx32):
    test_tensor_xi_statistics(H, ctx32, 128)


def test_tf32_matches_float32_path_and_differs_from_fp16(H, ctx32):
    """N = 256, 260 sequences, Dirichlet(0.1) rows: the TF32 recursion stays
    within the bounds of the float32 path, and its log-likelihoods are not
    the FP16 path's (the operand type really changed)."""
    from paper_2605_29208_gb300 import _lib
    models, values, offsets, mid, model, batch = build(H, ctx32, "diag_gauss", 256, 16, 0.1, [64] * 260, 1, 1250)
    ll2, g2, _ = H.forward_backward(ctx32, model, batch)
    ctx32.set_option(_lib.OPT_TENSOR_RECURRENCE, 1)
    ll1, _, _ = H.forward_backward(ctx32, model, batch)
    ctx32.set_option(_lib.OPT_TENSOR_RECURRENCE, 0)
    ll0, g0, _ = H.forward_backward(ctx32, model, batch)
    ll0, ll1, ll2 = ll0.cpu().numpy(), ll1.cpu().numpy(), ll2.cpu().numpy()
    assert np.all(np.abs(ll2 - ll0) <= TC_LL_RTOL * np.maximum(1.0, np.abs(ll0)))
    assert float((g2 - g0).abs().max()) <= TC_GAMMA_ATOL
    assert np.any(ll2 != ll1)
