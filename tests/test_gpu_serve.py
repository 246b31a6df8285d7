"""The request server (hmm_serve_*): continuous batching of decode,
posterior and fit requests.  Each request's result is the same run alone
(one slot, batches of one) and in a mix (four slots, batches of up to eight
requests of different lengths, admitted while others run), within the
parity tolerances, and matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth
from parity import check_viterbi_fp64

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4
PARAM_RTOL = 1e-4


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


def make_requests(n=30, seed=5):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        kind = ("decode", "posterior", "fit")[i % 3]
        family, D = (("gamma", 1), ("full_gauss", 3))[(i // 3) % 2]
        N = (4, 16, 64)[(i // 6) % 3]
        T = int(rng.integers(40, 300))
        truth = synth.small_models(family, N, 1, seed=1000 + i, D=D)[0]
        values, _, _ = synth.make_batch(2000 + i, [truth], [T], [0])
        if D > 1:
            values = values.reshape(-1, D)
        model = synth.perturb(np.random.default_rng(i), truth) if kind == "fit" else truth
        reqs.append(dict(kind=kind, model=model, values=values, n_iter=3 if kind == "fit" else 0))
    return reqs


def run(H, ctx, reqs, alone, **opts):
    srv = H.Server(ctx, **opts)
    try:
        out = []
        if alone:
            for r in reqs:
                t = srv.submit(r["kind"], r["model"], r["values"], r["n_iter"])
                out.append(srv.wait(t, 120000.0))
        else:
            ts = [srv.submit(r["kind"], r["model"], r["values"], r["n_iter"]) for r in reqs]
            out = [srv.wait(t, 120000.0) for t in ts]
        stats = srv.stats()
    finally:
        srv.close()
    return out, stats


def close_params(a, b, rtol):
    np.testing.assert_allclose(a["pi"], b["pi"], rtol=rtol, atol=1e-6)
    np.testing.assert_allclose(a["A"], b["A"], rtol=rtol, atol=1e-6)
    for k in b["params"]:
        np.testing.assert_allclose(a["params"][k], b["params"][k], rtol=rtol, atol=1e-6, err_msg=k)


def test_serve_alone_vs_mix(H, ctx):
    reqs = make_requests()
    alone, st1 = run(H, ctx, reqs, alone=True, n_slots=1, max_batch=1)
    mix, st2 = run(H, ctx, reqs, alone=False, n_slots=4, max_batch=8)
    assert st1["completed"] == len(reqs) and st2["completed"] == len(reqs)
    assert 0 < st2["p50_ms"] <= st2["p99_ms"]
    for r, a, m in zip(reqs, alone, mix):
        assert a["status"] == 0 and m["status"] == 0
        if r["kind"] == "decode":
            np.testing.assert_array_equal(a["path"], m["path"])
            assert abs(a["score"] - m["score"]) <= 1e-9 * max(1.0, abs(a["score"]))
        elif r["kind"] == "posterior":
            assert abs(a["loglik"] - m["loglik"]) <= LL_RTOL * max(1.0, abs(a["loglik"]))
            np.testing.assert_allclose(a["gamma"], m["gamma"], atol=GAMMA_ATOL, rtol=0)
        else:
            np.testing.assert_allclose(a["trace"], m["trace"], rtol=LL_RTOL)
            close_params(a["params"], m["params"], PARAM_RTOL)


def test_serve_matches_oracle(H, ctx):
    reqs = make_requests(n=12, seed=9)
    mix, _ = run(H, ctx, reqs, alone=False, n_slots=3, max_batch=4)
    for r, m in zip(reqs, mix):
        o = om(r["model"])
        y = np.asarray(r["values"], np.float64)
        if r["kind"] == "posterior":
            fb = O.forward_backward(o, y)
            assert abs(m["loglik"] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"]))
            np.testing.assert_allclose(m["gamma"], fb["gamma"], atol=GAMMA_ATOL)
        elif r["kind"] == "decode":
            check_viterbi_fp64(m["path"], m["score"], o, y, where="serve")
        else:
            ref_models, ref_trace = O.fit([o], y, np.array([0, len(y)]), np.zeros(1, np.int32), r["n_iter"])
            np.testing.assert_allclose(m["trace"], ref_trace[:, 0], rtol=LL_RTOL)
            g, ref = m["params"], ref_models[0]
            np.testing.assert_allclose(g["A"], ref.A, rtol=PARAM_RTOL, atol=1e-6)
            for k, v in ref.params.items():
                np.testing.assert_allclose(g["params"][k], v, rtol=PARAM_RTOL, atol=1e-6, err_msg=k)


def test_serve_admission_errors(H, ctx):
    from paper_2605_29208_gb300._lib import HmmError
    model = synth.small_models("gamma", 16, 1, seed=3)[0]
    values, _, _ = synth.make_batch(3, [model], [3000], [0])
    # a request larger than the whole budget is refused at submission
    srv = H.Server(ctx, n_slots=1, max_batch=1, mem_budget=1 << 20)
    with pytest.raises(HmmError) as e:
        srv.submit("posterior", model, values)
    assert e.value.status == 2
    srv.close()
    # a full queue answers HMM_E_BUSY while the only slot is occupied
    srv = H.Server(ctx, n_slots=1, max_batch=1, max_queue=2)
    long_vals, _, _ = synth.make_batch(4, [model], [20000], [0])
    tickets = [srv.submit("fit", model, long_vals, 30)]
    busy = False
    for _ in range(6):
        try:
            tickets.append(srv.submit("decode", model, values))
        except HmmError as err:
            assert err.status == 6
            busy = True
            break
    assert busy
    for t in tickets:
        assert srv.wait(t, 120000.0)["status"] == 0
    srv.close()
