"""Pins of the oracle's forward/backward, posteriors and Viterbi against
what the mathematics fixes: brute-force enumeration of all N^T paths,
invariants, and special cases that reduce to simpler closed forms."""
import numpy as np
import pytest
from scipy.special import logsumexp

from oracle import hmm_oracle as O


def rand_hmm(rng, N, T, zero_frac=0.0):
    pi = rng.dirichlet(np.ones(N))
    A = rng.dirichlet(np.ones(N), size=N)
    if zero_frac:
        mask = rng.random((N, N)) < zero_frac
        np.fill_diagonal(mask, False)
        A = np.where(mask, 0.0, A)
        A /= A.sum(1, keepdims=True)
    logb = rng.normal(-2, 3, (T, N))
    with np.errstate(divide="ignore"):
        return np.log(pi), np.log(A), logb


def test_lse_matches_library():
    rng = np.random.default_rng(0)
    x = rng.normal(0, 50, (7, 11))
    np.testing.assert_allclose(O.lse(x, 0), logsumexp(x, 0), rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(O.lse(x, 1), logsumexp(x, 1), rtol=1e-14, atol=1e-12)
    assert O.lse(np.array([-np.inf, -np.inf]), 0) == -np.inf


@pytest.mark.parametrize("N,T", [(1, 5), (2, 1), (2, 6), (3, 5), (2, 8), (3, 7)])
def test_forward_backward_vs_brute_force(N, T):
    rng = np.random.default_rng(100 * N + T)
    logpi, logA, logb = rand_hmm(rng, N, T)
    fb = O.forward_backward_logb(logpi, logA, logb)
    bf = O.brute_force(logpi, logA, logb)
    assert abs(fb["logL"] - bf["logL"]) <= 1e-11 * max(1, abs(bf["logL"]))
    np.testing.assert_allclose(fb["gamma"], bf["gamma"], atol=1e-12)
    np.testing.assert_allclose(fb["xi_sum"], bf["xi_sum"], atol=1e-12)


@pytest.mark.parametrize("N,T", [(2, 6), (3, 6), (3, 8)])
def test_structural_zeros_vs_brute_force(N, T):
    rng = np.random.default_rng(7 + N * T)
    logpi, logA, logb = rand_hmm(rng, N, T, zero_frac=0.4)
    fb = O.forward_backward_logb(logpi, logA, logb)
    bf = O.brute_force(logpi, logA, logb)
    assert abs(fb["logL"] - bf["logL"]) <= 1e-11 * max(1, abs(bf["logL"]))
    np.testing.assert_allclose(fb["gamma"], bf["gamma"], atol=1e-12)
    np.testing.assert_allclose(fb["xi_sum"], bf["xi_sum"], atol=1e-12)


@pytest.mark.parametrize("N,T", [(2, 7), (3, 6), (3, 8)])
def test_viterbi_vs_brute_force(N, T):
    rng = np.random.default_rng(1000 + N * T)
    logpi, logA, logb = rand_hmm(rng, N, T)
    q, score = O.viterbi_logb(logpi, logA, logb)
    bf = O.brute_force(logpi, logA, logb)
    assert abs(score - bf["map_score"]) <= 1e-11 * max(1, abs(score))
    np.testing.assert_array_equal(q, bf["map_path"])


def test_viterbi_tie_break_lowest_index():
    # two identical states: every path has the same score; the reading
    # keeps the lowest predecessor and the lowest final state -> all zeros
    N, T = 2, 5
    logpi = np.log(np.full(N, 0.5))
    logA = np.log(np.full((N, N), 0.5))
    logb = np.zeros((T, N))
    q, _ = O.viterbi_logb(logpi, logA, logb)
    np.testing.assert_array_equal(q, np.zeros(T, np.int32))
    q32, _ = O.viterbi_fp32(logpi, logA, logb)
    np.testing.assert_array_equal(q32, np.zeros(T, np.int32))


def test_invariants_long_sequence():
    rng = np.random.default_rng(5)
    N, T = 5, 400
    logpi, logA, logb = rand_hmm(rng, N, T)
    fb = O.forward_backward_logb(logpi, logA, logb)
    alpha, beta, logL = fb["alpha"], fb["beta"], fb["logL"]
    # forward logL equals the backward one
    lb = float(logsumexp(logpi + logb[0] + beta[0]))
    assert abs(lb - logL) <= 1e-10 * abs(logL)
    # every t gives the same total: sum_j alpha_t beta_t = P(y)
    tot = logsumexp(alpha + beta, axis=1)
    np.testing.assert_allclose(tot, logL, rtol=1e-12)
    g = fb["gamma"]
    np.testing.assert_allclose(g.sum(1), 1.0, atol=1e-12)
    # per-t xi marginals equal gamma
    for t in range(0, T - 1, 37):
        xi = np.exp(alpha[t][:, None] + logA + (logb[t + 1] + beta[t + 1])[None] - logL)
        np.testing.assert_allclose(xi.sum(1), g[t], atol=1e-12)
        np.testing.assert_allclose(xi.sum(0), g[t + 1], atol=1e-12)
    # sum over all xi = T - 1, and row sums = sum_{t<T} gamma
    np.testing.assert_allclose(fb["xi_sum"].sum(), T - 1, rtol=1e-12)
    np.testing.assert_allclose(fb["xi_sum"].sum(1), g[:-1].sum(0), rtol=1e-11)


def test_special_cases():
    rng = np.random.default_rng(9)
    T = 50
    # N = 1: logL = sum_t log b(y_t)
    logb = rng.normal(-1, 2, (T, 1))
    fb = O.forward_backward_logb(np.zeros(1), np.zeros((1, 1)), logb)
    assert abs(fb["logL"] - logb.sum()) < 1e-10
    # rows of A equal to pi: i.i.d. mixture, Viterbi = per-t argmax
    N = 4
    pi = rng.dirichlet(np.ones(N))
    logb = rng.normal(0, 2, (T, N))
    logA = np.tile(np.log(pi), (N, 1))
    fb = O.forward_backward_logb(np.log(pi), logA, logb)
    iid = logsumexp(np.log(pi)[None] + logb, axis=1).sum()
    assert abs(fb["logL"] - iid) < 1e-10 * abs(iid)
    q, _ = O.viterbi_logb(np.log(pi), logA, logb)
    np.testing.assert_array_equal(q, np.argmax(np.log(pi)[None] + logb, axis=1))
    # T = 1: logL = lse(log pi + log b(y_1))
    fb = O.forward_backward_logb(np.log(pi), logA, logb[:1])
    assert abs(fb["logL"] - logsumexp(np.log(pi) + logb[0])) < 1e-12
    assert fb["xi_sum"].sum() == 0


def test_no_underflow_long_T():
    # Sec. 3.2: log space works for any T; the product of 1e5 emissions is
    # far below the double range, logL stays finite
    rng = np.random.default_rng(11)
    N, T = 2, 100_000
    logb = rng.normal(-20, 1, (T, N))
    pi = np.array([0.5, 0.5])
    A = np.array([[0.9, 0.1], [0.2, 0.8]])
    alpha = O.forward_log(np.log(pi), np.log(A), logb)
    assert np.isfinite(alpha[-1]).all() and alpha[-1].max() < -1e6


def test_viterbi_fp32_mode_agrees_with_fp64_on_clear_margins():
    rng = np.random.default_rng(21)
    N, T = 6, 300
    logpi, logA, logb = rand_hmm(rng, N, T)
    q64, s64, gap, fgap = O.viterbi_gaps(logpi, logA, logb)
    q32, s32 = O.viterbi_fp32(logpi.astype(np.float32), logA.astype(np.float32),
                              logb.astype(np.float32))
    if np.min(gap[1:][np.isfinite(gap[1:])]) > 1e-3 and fgap > 1e-3:
        np.testing.assert_array_equal(q32, q64)
    assert abs(s32 - s64) < 1e-4 * abs(s64)


def test_viterbi_fp32_vs_brute_force_on_rounded_tables():
    rng = np.random.default_rng(33)
    for N, T in [(2, 8), (3, 7)]:
        logpi, logA, logb = rand_hmm(rng, N, T)
        l32 = [x.astype(np.float32) for x in (logpi, logA, logb)]
        bf = O.brute_force(*[x.astype(np.float64) for x in l32])
        q32, s32 = O.viterbi_fp32(*l32)
        np.testing.assert_array_equal(q32, bf["map_path"])
        assert abs(s32 - bf["map_score"]) < 1e-4 * max(1, abs(s32))


def test_posterior_decode_tie_lowest():
    g = np.array([[0.5, 0.5], [0.2, 0.8], [0.7, 0.3]])
    np.testing.assert_array_equal(O.posterior_decode(g), [0, 1, 0])


def grid_hmm(rng, N, T, step=0.125):
    """Log tables on a grid of multiples of `step` (small integers times a
    power of two), so that every float32 sum of a few of them is exact and
    float32 decoding equals exact decoding."""
    g = lambda shape, lo, hi: (rng.integers(lo, hi, shape) * step).astype(np.float32)
    return g(N, -24, 0), g((N, N), -24, 0), g((T, N), -40, 8)


@pytest.mark.parametrize("N,T", [(1, 4), (2, 1), (2, 2), (2, 5), (2, 8), (3, 3), (3, 6), (3, 7)])
def test_viterbi_fp32_mitm_vs_brute_force_on_exact_tables(N, T):
    """On grid tables float32 arithmetic is exact: the meet-in-the-middle
    decoder must return a path of the exact maximal score, and the unique
    maximiser whenever there is one."""
    rng = np.random.default_rng(1000 + 10 * N + T)
    for _ in range(20):
        l32 = grid_hmm(rng, N, T)
        bf = O.brute_force(*[x.astype(np.float64) for x in l32])
        q, s = O.viterbi_fp32_mitm(*l32)
        assert s == bf["map_score"]
        assert O.path_logprob(*[x.astype(np.float64) for x in l32], q) == bf["map_score"]
        if np.sum(bf["all_scores"] == bf["map_score"]) == 1:
            np.testing.assert_array_equal(q, bf["map_path"])


def test_viterbi_fp32_mitm_tie_rule_hand_example():
    """A worked example (computed by hand from the tie rules) where the
    two decoders return different maximisers.  N = 2, T = 3, log pi =
    (ln 1/2, ln 1/2), log A = [[-1, 0], [0, -1]], log b = 0: every
    alternating path scores ln 1/2.  One forward sweep ends in the lowest
    final state 0 and follows psi_2(0) = 1, psi_1(1) = 0: (0, 1, 0).  The
    meet-in-the-middle decoder (h = 1) has delta_1 = beta_1 = (0, 0) after
    shifting, so q_1 = 0; psi_1(0) = 1 and phi_1(0) = 1 give (1, 0, 1)."""
    lpi = np.log(np.array([0.5, 0.5])).astype(np.float32)
    lA = np.array([[-1.0, 0.0], [0.0, -1.0]], np.float32)
    lb = np.zeros((3, 2), np.float32)
    q, s = O.viterbi_fp32_mitm(lpi, lA, lb)
    np.testing.assert_array_equal(q, [1, 0, 1])
    q1, s1 = O.viterbi_fp32(lpi, lA, lb)
    np.testing.assert_array_equal(q1, [0, 1, 0])
    assert s == s1 == float(np.float32(np.log(0.5)))


def test_viterbi_fp32_mitm_special_cases():
    rng = np.random.default_rng(5)
    # T = 0 and T = 1
    for fn in (O.viterbi_fp32_mitm, O.viterbi_fp32):
        q, s = fn(np.zeros(3, np.float32), np.zeros((3, 3), np.float32), np.zeros((0, 3), np.float32))
        assert len(q) == 0 and s == 0.0
    lpi, lA, lb = grid_hmm(rng, 3, 1)
    q, s = O.viterbi_fp32_mitm(lpi, lA, lb)
    assert q[0] == int(np.argmax(lpi + lb[0])) and s == float((lpi + lb[0]).max())
    # rows of A equal to pi: i.i.d. mixture, the path is the per-t argmax
    N, T = 4, 41
    lpi = (rng.integers(-16, 0, N) * 0.25).astype(np.float32)
    lA = np.tile(lpi, (N, 1))
    lb = (rng.normal(0, 3, (T, N))).astype(np.float32)
    q, _ = O.viterbi_fp32_mitm(lpi, lA, lb)
    np.testing.assert_array_equal(q, np.argmax(lpi[None, :] + lb, axis=1))
    # a structural zero: the path never uses a forbidden transition
    with np.errstate(divide="ignore"):
        lA = np.log(np.array([[0.5, 0.5, 0], [0, 0.5, 0.5], [0.5, 0, 0.5]])).astype(np.float32)
    lb = rng.normal(0, 2, (30, 3)).astype(np.float32)
    q, s = O.viterbi_fp32_mitm(np.log(np.ones(3) / 3).astype(np.float32), lA, lb)
    assert np.isfinite(s) and np.all(np.isfinite(lA[q[:-1], q[1:]]))


def test_viterbi_fp32_mitm_agrees_with_fp64_on_clear_margins():
    rng = np.random.default_rng(22)
    for N, T in [(6, 300), (16, 501), (3, 1000)]:
        logpi, logA, logb = rand_hmm(rng, N, T)
        q64, s64, gap, fgap = O.viterbi_gaps(logpi, logA, logb)
        q32, s32 = O.viterbi_fp32_mitm(logpi.astype(np.float32), logA.astype(np.float32),
                                       logb.astype(np.float32))
        assert abs(s32 - s64) < 1e-5 * abs(s64)
        gap_of_path = s64 - O.path_logprob(logpi, logA, logb, q32)
        assert -1e-10 * abs(s64) <= gap_of_path < 1e-4


@pytest.mark.parametrize("N,T", [(2, 1), (2, 6), (3, 5), (3, 7)])
def test_path_logprob_vs_brute_force(N, T):
    rng = np.random.default_rng(200 + 10 * N + T)
    logpi, logA, logb = rand_hmm(rng, N, T)
    bf = O.brute_force(logpi, logA, logb)
    got = np.array([O.path_logprob(logpi, logA, logb, p) for p in bf["paths"]])
    np.testing.assert_allclose(got, bf["all_scores"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,T", [(2, 6), (3, 5), (3, 7)])
def test_viterbi_gaps_vs_brute_force_second_best(N, T):
    """step_gap[t, j] is the best score of a prefix ending in state j at t
    minus the best score of such a prefix whose state at t-1 is not
    psi_t(j); final_gap is the best path score minus the best score of a
    path ending in another state.  Both by enumeration."""
    rng = np.random.default_rng(300 + 10 * N + T)
    logpi, logA, logb = rand_hmm(rng, N, T)
    q, s, gap, fgap = O.viterbi_gaps(logpi, logA, logb)
    for t in range(1, T):
        bf = O.brute_force(logpi, logA, logb[:t + 1])
        P, sc = bf["paths"], bf["all_scores"]
        for j in range(N):
            sel = P[:, t] == j
            best_by_prev = np.array([sc[sel & (P[:, t - 1] == i)].max() for i in range(N)])
            order = np.sort(best_by_prev)
            assert abs(gap[t, j] - (order[-1] - order[-2])) < 1e-11
    bf = O.brute_force(logpi, logA, logb)
    best_by_last = np.array([bf["all_scores"][bf["paths"][:, -1] == j].max() for j in range(N)])
    order = np.sort(best_by_last)
    assert abs(fgap - (order[-1] - order[-2])) < 1e-11
    np.testing.assert_array_equal(q, bf["map_path"])
