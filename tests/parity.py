"""Shared parity checks of the GPU tests against the oracle.

Viterbi (Sec. 3.3, Eq. 3-4):
  * against the float32-mode oracle on the float32 log-emission table the
    device decoded from, bit for bit: the meet-in-the-middle order for
    padded state counts up to 32 (the small-N decoder), the single forward
    sweep above (the large-N decoder);
  * against the float64 oracle: the score within 1e-5 relative, and the
    path identical except at a near-tie, where the float64 log-probability
    of the device's path must lie within VIT_SCORE_GAP of the float64
    optimum.  Every such site is recorded in NEAR_TIES (printed at the end
    of the session).

M-step parameters: 1e-4 relative (PARAM_RTOL) for one iteration from the
same parameters; iterated fits are checked one iteration at a time, each
from the device's own previous parameters (check_fit_iterations)."""
import numpy as np

from oracle import hmm_oracle as O

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4
PARAM_RTOL = 1e-4
VIT_SCORE_GAP = 1e-4
NEAR_TIES = []


def om(d):
    return O.Model(d["family"], np.array(d["pi"], copy=True), np.array(d["A"], copy=True),
                   {k: np.array(v, copy=True) for k, v in d["params"].items()}, tuple(d.get("components", ())))


def _logs(o):
    with np.errstate(divide="ignore"):
        return np.log(o.pi), np.log(o.A)


def small_decoder(N):
    """True when the device decodes N states with the meet-in-the-middle
    small-N kernel (padded N <= 32)."""
    return N <= 32


def check_viterbi_fp64(path, score, o, y, where=None):
    """Device path / score of one sequence against the float64 oracle."""
    logpi, logA = _logs(o)
    logb = O.emission_logpdf(o, np.asarray(y, np.float64))
    q, sc = O.viterbi_logb(logpi, logA, logb)
    path = np.asarray(path)
    assert abs(score - sc) <= LL_RTOL * max(1.0, abs(sc)), (where, score, sc)
    if not np.array_equal(path, q):
        gap = sc - O.path_logprob(logpi, logA, logb, path)
        assert np.isfinite(gap) and gap < VIT_SCORE_GAP, (where, gap)
        NEAR_TIES.append((where, int(np.sum(path != q)), float(gap)))


def check_viterbi_fp32(path, score, logpi32, logA32, logb32, N, where=None):
    """Device path of one sequence decoded from a float32 table: bit for
    bit equal to the float32-mode oracle of the decoder that ran."""
    fn = O.viterbi_fp32_mitm if small_decoder(N) else O.viterbi_fp32
    q, sc = fn(logpi32, logA32, logb32)
    np.testing.assert_array_equal(np.asarray(path), q, err_msg=str(where))
    assert abs(score - sc) <= LL_RTOL * max(1.0, abs(sc)), (where, score, sc)


def check_viterbi_table_batch(H, ctx, model, batch, models, values, offsets, mid, path, score):
    """For table families (and every family at N > 32): the decode is a
    function of the float32 table hmm_emission_logpdf returns and of the
    float32 log pi / log A, so it must equal the float32-mode oracle on it."""
    lb = H.emission_logpdf(ctx, model, batch).cpu().numpy()
    for s in range(len(offsets) - 1):
        o = om(models[mid[s]])
        lpi, lA = _logs(o)
        check_viterbi_fp32(path[offsets[s]:offsets[s + 1]], score[s], lpi.astype(np.float32),
                           lA.astype(np.float32), lb[offsets[s]:offsets[s + 1]], o.n_states, where=s)


def assert_params_close(got, ref, rtol=PARAM_RTOL, atol=1e-7):
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g["pi"], r.pi, rtol=rtol, atol=max(atol, 1e-6))
        np.testing.assert_allclose(g["A"], r.A, rtol=rtol, atol=max(atol, 1e-6))
        for k, v in r.params.items():
            gv = np.asarray(g["params"][k])
            if r.family == "vonmises" and k == "mu":
                np.testing.assert_allclose(np.angle(np.exp(1j * (gv - v))), 0, atol=rtol)
            else:
                np.testing.assert_allclose(gv, v, rtol=rtol, atol=atol, err_msg=f"{r.family}.{k}")


def check_fit_iterations(H, ctx, model, batch, values, offsets, mid, n_iter, rtol=PARAM_RTOL, atol=1e-7,
                         nu_mode="ecm", **fit_kw):
    """n_iter Baum-Welch iterations on the device, one hmm_fit call each.
    Iteration k is checked against the oracle's iteration applied to the
    device's parameters entering k (logL of those parameters within
    LL_RTOL, new parameters within rtol), so each comparison measures one
    M-step's error and none compounds.  Returns the device trace [n_iter]
    and the oracle's compounded fit from the same start, for callers that
    also bound the compounded drift."""
    start = [om(m) for m in model.get()]
    trace = []
    for k in range(n_iter):
        before = [om(m) for m in model.get()]
        tr, done = H.fit(ctx, model, batch, n_iter=1, **fit_kw)
        assert done == 1
        ref, ll = O.em_iteration(before, values, offsets, mid, nu_mode=nu_mode)
        M = len(before)
        ref_ll = np.array([ll[np.asarray(mid) == m].sum() for m in range(M)])
        np.testing.assert_allclose(tr[0, :M], ref_ll, rtol=LL_RTOL, err_msg=f"iteration {k}")
        assert_params_close(model.get(), ref, rtol=rtol, atol=atol)
        trace.append(tr[0, :M])
    return np.array(trace), O.fit(start, values, offsets, mid, n_iter, nu_mode=nu_mode)
