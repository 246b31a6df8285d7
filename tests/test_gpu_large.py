"""Parity of the large-N path (padded N = 64 ... 1024: float32 CUDA cores,
groups of sequences in lock step, xi as a blocked outer-product sum) with
the FP64 oracle.  Same bar as the small-N path: per-sequence logL 1e-5
relative, occupancies 1e-4 absolute, M-step parameters 1e-4 relative,
Viterbi bit-identical to the float32-mode oracle on a shared table."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import check_fit_iterations, check_viterbi_fp32, check_viterbi_fp64, check_viterbi_table_batch

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4
PARAM_RTOL = 1e-4

LENGTHS = [1, 2, 0, 37, 130, 9, 64, 65, 11, 3]


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


@pytest.fixture(scope="module")
def ctx(H):
    return H.Context(0)


def om(d):
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(),
                   {k: np.array(v, copy=True) for k, v in d["params"].items()})


def check_fb(ll, gamma, models, values, offsets, mid, xi_ref=None):
    for s in range(len(offsets) - 1):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            assert ll[s] == 0.0
            continue
        fb = O.forward_backward(om(models[mid[s]]), np.asarray(y, np.float64))
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"])), (s, ll[s], fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL, rtol=0)


@pytest.mark.parametrize("family,N,conc", [("gauss", 33, 1.0), ("gauss", 64, 1.0), ("poisson", 100, 1.0),
                                           ("gamma", 200, 1.0), ("gauss", 128, 0.1), ("vonmises", 300, 1.0)])
def test_large_forward_backward(H, ctx, family, N, conc):
    models = synth.small_models(family, N, 2, seed=600 + N, conc=conc)
    mid = np.arange(len(LENGTHS)) % 2
    values, offsets, mid = synth.make_batch(610 + N, models, LENGTHS, mid)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    ll, gamma, path = H.forward_backward(ctx, model, batch, want_path=True)
    check_fb(ll.cpu().numpy(), gamma.cpu().numpy(), models, values, offsets, mid)


def test_large_forward_backward_512_sparse(H, ctx):
    """N = 512 with Dirichlet(0.1) rows (many transition probabilities far
    below float32's normal range) and diagonal Gaussian emissions, D = 4."""
    models = synth.small_models("diag_gauss", 512, 1, seed=5, conc=0.1, D=4)
    lengths = [1, 40, 0, 97]
    values, offsets, mid = synth.make_batch(15, models, lengths, np.zeros(len(lengths), np.int32))
    values = values.reshape(-1, 4)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid, dim=4)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    check_fb(ll.cpu().numpy(), gamma.cpu().numpy(), models, values, offsets, mid)


@pytest.mark.parametrize("N", [64, 96, 256, 1024])
def test_large_table_mode_xi(H, ctx, N):
    """A shared float32 log b table: logL, gamma and the statistics'
    transition sums against the oracle's xi."""
    import torch
    rng = np.random.default_rng(N)
    models = synth.small_models("gauss", N, 1, seed=N, conc=0.5)
    lengths = [1, 2, 17, 70] if N < 1024 else [1, 9, 23]
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    logb = rng.normal(-3, 2, (offsets[-1], N)).astype(np.float32)
    mid = np.zeros(len(lengths), np.int32)
    model = H.Model(ctx, models)
    batch = H.Batch(np.zeros(offsets[-1]), offsets, mid)
    ll, gamma, _ = H.forward_backward(ctx, model, batch, logb=torch.as_tensor(logb).cuda())
    ll = ll.cpu().numpy()
    gamma = gamma.cpu().numpy()
    m = om(models[0])
    for s in range(len(lengths)):
        fb = O.forward_backward_logb(np.log(m.pi), np.log(m.A), logb[offsets[s]:offsets[s + 1]].astype(np.float64))
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"]))
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL)


def oracle_stats(models, values, offsets, mid):
    out = []
    for m, model in enumerate(models):
        o = om(model)
        N = len(model["pi"])
        idx = [s for s in range(len(offsets) - 1) if mid[s] == m]
        g1, xi, ll = np.zeros(N), np.zeros((N, N)), 0.0
        cols = np.zeros((N, 3))
        for s in idx:
            y = np.asarray(values[offsets[s]:offsets[s + 1]], np.float64)
            if len(y) == 0:
                continue
            fb = O.forward_backward(o, y)
            ll += fb["logL"]
            g1 += fb["gamma"][0]
            xi += fb["xi_sum"]
            w = fb["gamma"]
            cols += np.stack([w.sum(0), (w * y[:, None]).sum(0), (w * y[:, None] ** 2).sum(0)], axis=1)
        out.append(np.concatenate([[len(idx), ll], g1, xi.ravel(), cols.ravel()]))
    return np.concatenate(out)


@pytest.mark.parametrize("N", [40, 128])
def test_large_estep_stats(H, ctx, N):
    models = synth.small_models("gauss", N, 2, seed=700 + N)
    lengths = [50, 3, 0, 200, 120, 1, 77]
    values, offsets, mid = synth.make_batch(701, models, lengths, np.arange(len(lengths)) % 2)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    got = stats.get()
    ref = oracle_stats(models, values, offsets, mid)
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=2e-4)


def assert_params_close(got_models, ref_models, rtol):
    for g, r in zip(got_models, ref_models):
        np.testing.assert_allclose(g["pi"], r.pi, rtol=rtol, atol=1e-6)
        np.testing.assert_allclose(g["A"], r.A, rtol=rtol, atol=1e-6)
        for k, v in r.params.items():
            np.testing.assert_allclose(g["params"][k], v, rtol=rtol, atol=1e-6, err_msg=f"{r.family}.{k}")


@pytest.mark.parametrize("family,N,D", [("gauss", 40, 1), ("gamma", 70, 1), ("student_t", 64, 1),
                                        ("diag_gauss", 64, 3), ("full_gauss", 33, 3)])
def test_large_mstep(H, ctx, family, N, D):
    truth = synth.small_models(family, N, 2, seed=800 + N, D=D)
    lengths = [400, 250, 1, 333, 128, 90]
    values, offsets, mid = synth.make_batch(801, truth, lengths, np.arange(len(lengths)) % 2)
    if D > 1:
        values = values.reshape(-1, D)
    rng = np.random.default_rng(7)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid, dim=D)
    stats, _ = H.estep_stats(ctx, model, batch)
    H.mstep(ctx, model, stats, batch=batch)
    ref, _ = O.em_iteration([om(m) for m in init], np.asarray(values, np.float64), offsets, mid)
    assert_params_close(model.get(), ref, PARAM_RTOL)


def test_large_fit(H, ctx):
    truth = synth.small_models("gauss", 48, 1, seed=901)
    lengths = [300, 200, 150, 64]
    values, offsets, mid = synth.make_batch(902, truth, lengths, np.zeros(len(lengths), np.int32))
    rng = np.random.default_rng(8)
    init = [synth.perturb(rng, t) for t in truth]
    model = H.Model(ctx, init)
    batch = H.Batch(values, offsets, mid)
    trace, (ref_models, ref_trace) = check_fit_iterations(H, ctx, model, batch, values, offsets, mid, 3)
    np.testing.assert_allclose(trace[:, 0], ref_trace.sum(axis=1), rtol=LL_RTOL)
    assert_params_close(model.get(), ref_models, PARAM_RTOL)


@pytest.mark.parametrize("N", [64, 100, 256, 600])
def test_large_viterbi_bit_exact_table(H, ctx, N):
    import torch
    rng = np.random.default_rng(50 + N)
    models = synth.small_models("gauss", N, 1, seed=N, conc=0.5)
    lengths = [1, 2, 5, 64, 65, 129, 300]
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    logb = rng.normal(-2, 2, (offsets[-1], N)).astype(np.float32)
    logb[10:20] = np.round(logb[10:20])       # exact ties
    mid = np.zeros(len(lengths), np.int32)
    model = H.Model(ctx, models)
    batch = H.Batch(np.zeros(offsets[-1]), offsets, mid)
    path, score = H.viterbi(ctx, model, batch, logb=torch.as_tensor(logb).cuda())
    path = path.cpu().numpy()
    score = score.cpu().numpy()
    m = models[0]
    lpi = np.log(m["pi"]).astype(np.float32)
    lA = np.log(m["A"]).astype(np.float32)
    for s in range(len(lengths)):
        check_viterbi_fp32(path[offsets[s]:offsets[s + 1]], score[s], lpi, lA, logb[offsets[s]:offsets[s + 1]], N,
                           where=s)


@pytest.mark.parametrize("family,N", [("gauss", 70), ("poisson", 128)])
def test_large_viterbi_vs_fp64(H, ctx, family, N):
    models = synth.small_models(family, N, 2, seed=61 + N)
    lengths = [1, 2, 40, 200, 0, 77]
    values, offsets, mid = synth.make_batch(17, models, lengths, np.arange(len(lengths)) % 2)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    path, score = H.viterbi(ctx, model, batch)
    path = path.cpu().numpy()
    score = score.cpu().numpy()
    for s in range(len(lengths)):
        y = values[offsets[s]:offsets[s + 1]]
        if len(y) == 0:
            assert score[s] == 0.0
            continue
        o = om(models[mid[s]])
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], o, y, where=(family, N, s))
    check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score)


def test_large_weibull_mstep_unsupported(H, ctx):
    models = synth.small_models("weibull", 40, 1, seed=3)
    values, offsets, mid = synth.make_batch(3, models, [30, 20], np.zeros(2, np.int32))
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    with pytest.raises(Exception):
        H.mstep(ctx, model, stats, batch=batch)


@pytest.mark.parametrize("n_seq", [1, 9, 300])
def test_large_256_cluster_and_group_paths(H, ctx, n_seq):
    """Padded N = 256 runs on clusters of two CTAs with A in shared memory
    for up to 32 sequence groups (1 and 9 sequences here) and on the
    one-block kernels above that (300 sequences, 38 groups): both against
    the oracle (logL, gamma, Viterbi bit-exact on the float32 table and
    against float64)."""
    models = synth.small_models("gauss", 230, 1, seed=1234, conc=0.5)
    rng = np.random.default_rng(n_seq)
    lengths = list(rng.integers(1, 400, n_seq)) if n_seq > 1 else [2500]
    values, offsets, mid = synth.make_batch(5 + n_seq, models, lengths, [0] * n_seq)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    ll, gamma = ll.cpu().numpy(), gamma.cpu().numpy()
    path, score = H.viterbi(ctx, model, batch)
    path, score = path.cpu().numpy(), score.cpu().numpy()
    o = om(models[0])
    for s in sorted({0, n_seq // 2, n_seq - 1}):
        y = values[offsets[s]:offsets[s + 1]]
        fb = O.forward_backward(o, y)
        assert abs(ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"])), (s, ll[s], fb["logL"])
        np.testing.assert_allclose(gamma[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL)
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], o, y, where=("N230", n_seq, s))
    check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score)


@pytest.mark.parametrize("N,lengths", [(230, [2500, 1, 2, 700, 33]), (129, [64, 65, 300]), (256, [1000, 5]),
                                       (40, [3000, 1, 17]), (100, [1500, 2, 64, 128])])
def test_large_single_sequence_groups(H, ctx, N, lengths):
    """Padded N = 64, 128, 256 with one sequence per model (the request
    server's case) run the single-sequence cluster kernels (64 columns per
    CTA, per-CTA power-of-two shifts joined exactly, st.async vector
    exchange).  logL and gamma per sequence against the oracle, the
    statistics record against the oracle's sums (their xi is formed from the
    stored forward / backward rows), Viterbi bit-identical to the
    float32-mode oracle on the shared table and against float64."""
    M = len(lengths)
    models = synth.small_models("gauss", N, M, seed=4321 + N, conc=0.5)
    mid = np.arange(M)
    values, offsets, mid = synth.make_batch(17 + N, models, lengths, mid)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    ll, gamma, _ = H.forward_backward(ctx, model, batch)
    check_fb(ll.cpu().numpy(), gamma.cpu().numpy(), models, values, offsets, mid)
    stats, _ = H.estep_stats(ctx, model, batch)
    np.testing.assert_allclose(stats.get(), oracle_stats(models, values, offsets, mid), rtol=2e-5, atol=2e-4)
    path, score = H.viterbi(ctx, model, batch)
    path, score = path.cpu().numpy(), score.cpu().numpy()
    for s in range(M):
        y = values[offsets[s]:offsets[s + 1]]
        check_viterbi_fp64(path[offsets[s]:offsets[s + 1]], score[s], om(models[s]), y, where=("single", N, s))
    check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score)
