"""CPU checks of two reformulations the CUDA path uses (no GPU, float64):

* meet-in-the-middle Viterbi: a forward max-plus sweep to h = floor(T/2), the
  max-plus backward recursion down to h, joined at the best state of h, then
  the two tracebacks, reproduce the oracle's maximum score and a path that
  attains it (brute force on tiny cases);
* time-parallel forward-backward: chunk products of the step matrices, a walk
  over the chunk boundaries, then every chunk rerun from its boundary vector,
  reproduce the oracle's posteriors and log-likelihood for chunk lengths that
  do and do not divide T, with T shorter than one chunk, and T = 1.

Both are written here with the same conventions as the kernels (rows scaled
by their maximum, logarithms of the scales carried separately) but share no
code with them."""
import numpy as np
import pytest

from oracle import hmm_oracle as O


def rand_hmm(rng, N, T):
    logpi = np.log(rng.dirichlet(np.ones(N)))
    logA = np.log(rng.dirichlet(np.ones(N), size=N))
    logb = rng.normal(0.0, 2.0, size=(T, N))
    return logpi, logA, logb


def viterbi_meet_in_middle(logpi, logA, logb):
    T, N = logb.shape
    h = T // 2
    ptr = np.zeros((T, N), np.int64)
    d = logpi + logb[0]
    for t in range(1, h + 1):                       # forward: psi_t in row t
        c = d[:, None] + logA
        ptr[t] = np.argmax(c, axis=0)
        d = c.max(axis=0) + logb[t]
    beta = np.zeros(N)
    for t in range(T - 2, h - 1, -1):               # backward: phi_t in row t + 1
        c = logA + (logb[t + 1] + beta)[None, :]
        ptr[t + 1] = np.argmax(c, axis=1)
        beta = c.max(axis=1)
    comb = d + beta
    q = np.zeros(T, np.int64)
    q[h] = int(np.argmax(comb))
    for t in range(h, 0, -1):
        q[t - 1] = ptr[t][q[t]]
    for t in range(h + 1, T):
        q[t] = ptr[t][q[t - 1]]
    return q, float(comb.max())


def path_score(logpi, logA, logb, q):
    return logpi[q[0]] + logb[0, q[0]] + sum(logA[q[t - 1], q[t]] + logb[t, q[t]] for t in range(1, len(q)))


@pytest.mark.parametrize("N,T", [(1, 5), (2, 1), (2, 2), (3, 3), (3, 7), (4, 8), (6, 101), (16, 400)])
def test_meet_in_the_middle_viterbi(N, T):
    rng = np.random.default_rng(100 * N + T)
    logpi, logA, logb = rand_hmm(rng, N, T)
    q, sc = viterbi_meet_in_middle(logpi, logA, logb)
    q_ref, sc_ref = O.viterbi_logb(logpi, logA, logb)
    assert abs(sc - sc_ref) <= 1e-9 * max(1.0, abs(sc_ref))
    assert abs(path_score(logpi, logA, logb, q) - sc_ref) <= 1e-9 * max(1.0, abs(sc_ref))
    if N ** T <= 5000:
        assert abs(O.brute_force(logpi, logA, logb)["map_score"] - sc) <= 1e-9 * max(1.0, abs(sc))


def _scaled(x):
    m = x.max()
    return x / m, np.log(m)


def forward_backward_chunked(logpi, logA, logb, L):
    """Posteriors and logL by the three-stage chunked scheme."""
    T, N = logb.shape
    A = np.exp(logA)
    cs = [(t0, min(t0 + L, T)) for t0 in range(0, T, L)]
    mb = logb.max(axis=1, keepdims=True)
    b = np.exp(logb - mb)                           # b_t scaled by its row maximum
    # 1. transfer matrices, rows scaled (log scales per row)
    Qf, ef, Qb, eb = [], [], [], []
    for c, (t0, t1) in enumerate(cs):
        lo = 1 if c == 0 else t0                    # forward skips t = 0
        hi = T - 1 if c == len(cs) - 1 else t1      # backward skips t = T - 1
        X, e = np.eye(N), np.zeros(N)
        for t in range(lo, t1):
            X = (X @ A) * b[t][None, :]
            s = X.max(axis=1)
            X, e = X / s[:, None], e + np.log(s) + mb[t, 0]
        Qf.append(X), ef.append(e)
        X, e = np.eye(N), np.zeros(N)
        for t in range(t0, hi):
            X = (X * b[t][None, :]) @ A
            s = X.max(axis=1)
            X, e = X / s[:, None], e + np.log(s) + mb[t, 0]
        Qb.append(X), eb.append(e)
    # 2. boundary walk: forward vector at the last step of each chunk,
    # backward z = b .* beta at the first step of each chunk
    vf, of = [None] * len(cs), [0.0] * len(cs)
    w, o = _scaled(np.exp(logpi + logb[0] - (logpi + logb[0]).max()))
    o += (logpi + logb[0]).max()
    for c in range(len(cs)):
        g = np.log(np.where(w > 0, w, 1e-300)) + ef[c]
        G = g.max()
        w = np.exp(g - G) @ Qf[c]
        w, s = _scaled(w)
        o += G + s
        vf[c], of[c] = w, o
    vb, ob = [None] * len(cs), [0.0] * len(cs)
    w, o = b[T - 1], mb[T - 1, 0]
    w, s = _scaled(w)
    o += s
    for c in range(len(cs) - 1, -1, -1):
        d = Qb[c] @ w
        g = np.log(np.where(d > 0, d, 1e-300)) + eb[c]
        G = g.max()
        w, s = _scaled(np.exp(g - G))
        o += G + s
        vb[c], ob[c] = w, o
    # 3. every chunk from its boundary vector: log alpha and log beta rows
    la, lb = np.zeros((T, N)), np.zeros((T, N))
    for c, (t0, t1) in enumerate(cs):
        if c == 0:
            v = np.exp(logpi + logb[0] - (logpi + logb[0]).max())
            o = (logpi + logb[0]).max()
            la[0] = np.log(v) + o
            t = 1
        else:
            v, o, t = vf[c - 1], of[c - 1], t0
        for t in range(t, t1):
            v = (v @ A) * b[t]
            v, s = _scaled(v)
            o += s + mb[t, 0]
            la[t] = np.log(v) + o
        if c == len(cs) - 1:
            lb[T - 1] = 0.0
            z, o = _scaled(b[T - 1])
            o += mb[T - 1, 0]
            t = T - 2
        else:
            z, o, t = vb[c + 1], ob[c + 1], t1 - 1
        for t in range(t, t0 - 1, -1):
            beta = A @ z
            lb[t] = np.log(beta) + o
            z, s = _scaled(b[t] * beta)
            o += s + mb[t, 0]
    lg = la + lb
    logL = O.lse(lg[0], axis=0)
    return np.exp(lg - logL), float(logL)


@pytest.mark.parametrize("N,T,L", [(2, 1, 4), (3, 5, 8), (3, 16, 4), (4, 17, 4), (5, 100, 7), (8, 257, 16),
                                   (16, 300, 64), (2, 1000, 32)])
def test_time_parallel_scheme(N, T, L):
    rng = np.random.default_rng(7 * N + T + L)
    logpi, logA, logb = rand_hmm(rng, N, T)
    gamma, logL = forward_backward_chunked(logpi, logA, logb, L)
    fb = O.forward_backward_logb(logpi, logA, logb)
    assert abs(logL - fb["logL"]) <= 1e-10 * max(1.0, abs(fb["logL"]))
    np.testing.assert_allclose(gamma, fb["gamma"], atol=1e-10, rtol=0)
