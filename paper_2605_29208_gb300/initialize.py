"""Starting parameters for Baum-Welch from the data: seeded k-means++.

The paper names k-means++ initialisation without constants; this module
fixes one reading (it is an input to the fit, not a parity target, and both
the CUDA path and the CPU checker receive its output as their starting
model):

* uniforms u_0..u_{N-1} from numpy ``default_rng(seed)``; the first centre
  is observation floor(u_0 T), centre j the first observation whose running
  sum of squared distances to the nearest centre so far exceeds u_j times
  the total (floor(u_j T) when the total is 0);
* Lloyd iterations until no assignment changes or 100 passes, ties to the
  lowest cluster index, an empty cluster keeps its centre;
* state j's emission from cluster j by moments (Gaussian mean / variance,
  Poisson mean, Gamma and Beta method of moments, ...), variances floored;
* pi uniform, A from the label transitions inside each sequence with one
  added to every count (add-one smoothing), rows normalised.

With a context the seeding and the Lloyd iterations run on the GPU
(hmm_kmeans, every restart of ``kmeanspp_init_many`` in one call); without
one, a host numpy version of the same rules runs.  The moments and the
label transitions are host numpy over the labels.
"""
from __future__ import annotations

import math

import numpy as np

VAR_FLOOR = 1e-6
MAX_ITER = 100


def _uniforms(seed, N):
    return np.random.default_rng(seed).random(N)


def _kmeanspp_host(X, u, max_iter=MAX_ITER):
    T = X.shape[0]
    K = len(u)
    C = np.empty((K, X.shape[1]))
    C[0] = X[min(int(math.floor(u[0] * T)), T - 1)]
    d2 = np.sum((X - C[0]) ** 2, axis=1)
    for j in range(1, K):
        tot = float(d2.sum())
        if tot > 0:
            i = min(int(np.searchsorted(np.cumsum(d2), u[j] * tot, side="right")), T - 1)
        else:
            i = min(int(math.floor(u[j] * T)), T - 1)
        C[j] = X[i]
        d2 = np.minimum(d2, np.sum((X - C[j]) ** 2, axis=1))
    labels = None
    for _ in range(max_iter):
        new = np.argmin(np.sum((X[:, None, :] - C[None, :, :]) ** 2, axis=2), axis=1)
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for j in range(K):
            sel = labels == j
            if sel.any():
                C[j] = X[sel].mean(axis=0)
    return C, labels


def _state_params(family, x, D):
    """Moment estimates of one cluster's emission parameters."""
    if len(x) == 0:
        x = np.zeros((1, D))
    if family == "gauss":
        return dict(mu=x[:, 0].mean(), sigma2=max(x[:, 0].var(), VAR_FLOOR))
    if family == "poisson":
        return dict(lam=max(x[:, 0].mean(), 1e-3))
    if family == "gamma":
        m, v = x[:, 0].mean(), max(x[:, 0].var(), VAR_FLOOR)
        return dict(alpha=max(m * m / v, 1e-3), beta=max(m / v, 1e-6))
    if family == "beta":
        m, v = x[:, 0].mean(), max(x[:, 0].var(), VAR_FLOOR)
        c = max(m * (1 - m) / v - 1, 1e-3)
        return dict(a=max(m * c, 1e-3), b=max((1 - m) * c, 1e-3))
    if family == "weibull":
        m, s = x[:, 0].mean(), max(x[:, 0].std(), 1e-3)
        k = max(min((s / max(m, 1e-6)) ** -1.086, 50.0), 0.1)   # Justus' approximation
        return dict(k=k, lam=max(m, 1e-6))
    if family == "negbin":
        m, v = x[:, 0].mean(), x[:, 0].var()
        r = m * m / (v - m) if v > m else 1e3
        return dict(r=max(r, 1e-3), p=r / (r + max(m, 1e-9)))
    if family == "student_t":
        return dict(mu=x[:, 0].mean(), sigma2=max(x[:, 0].var(), VAR_FLOOR), nu=10.0)
    if family == "vonmises":
        c, s = np.cos(x[:, 0]).mean(), np.sin(x[:, 0]).mean()
        R = min(np.hypot(c, s), 0.999)
        kappa = R * (2 - R * R) / (1 - R * R)                    # Banerjee et al. approximation
        return dict(mu=np.arctan2(s, c), kappa=max(kappa, 1e-3))
    if family == "diag_gauss":
        return dict(mu=x.mean(axis=0), var=np.maximum(x.var(axis=0), VAR_FLOOR))
    if family == "full_gauss":
        cov = np.cov(x.T, bias=True).reshape(D, D) if len(x) > 1 else np.eye(D)
        return dict(mu=x.mean(axis=0), cov=cov + VAR_FLOOR * np.eye(D))
    raise ValueError(family)


def _features(family, values):
    X = np.asarray(values, np.float64)
    X = X[:, None] if X.ndim == 1 else X
    feat = X
    if family == "vonmises":        # cluster angles on the unit circle
        feat = np.stack([np.cos(X[:, 0]), np.sin(X[:, 0])], axis=1)
    # the device clusters float32 features: round them once for both routes
    return X, feat.astype(np.float32).astype(np.float64)


def _model_from_labels(family, N, X, centres, labels, offsets):
    D = X.shape[1]
    # order the states by their first centre coordinate (a stable labelling)
    order = np.argsort(centres[:, 0], kind="stable")
    rank = np.empty(N, np.int64)
    rank[order] = np.arange(N)
    labels = rank[np.asarray(labels, np.int64)]
    per = [_state_params(family, X[labels == j], D) for j in range(N)]
    params = {k: np.array([p[k] for p in per]) for k in per[0]}
    counts = np.ones((N, N))
    offsets = np.asarray(offsets, np.int64)
    for s in range(len(offsets) - 1):
        lab = labels[offsets[s]:offsets[s + 1]]
        if len(lab) > 1:
            np.add.at(counts, (lab[:-1], lab[1:]), 1.0)
    A = counts / counts.sum(axis=1, keepdims=True)
    return dict(family=family, pi=np.full(N, 1.0 / N), A=A, params=params)


def kmeanspp_init_many(ctx, family, N, values, offsets, seeds):
    """Starting models of several restarts (one per seed) with one device
    k-means++ call for all of them (hmm_kmeans)."""
    from . import kmeans
    X, feat = _features(family, values)
    u = np.stack([_uniforms(s, N) for s in seeds])
    C, lab, _ = kmeans(ctx, feat.astype(np.float32), u, max_iter=MAX_ITER)
    C, lab = C.cpu().numpy(), lab.cpu().numpy()
    return [_model_from_labels(family, N, X, C[r], lab[r], offsets) for r in range(len(seeds))]


def kmeanspp_init(family, N, values, offsets, seed=0, ctx=None):
    """Starting model dict for `family` with N states from the packed
    observations (values [total_T] or [total_T, D], offsets [S+1]); on the
    GPU when a context is given."""
    if ctx is not None:
        return kmeanspp_init_many(ctx, family, N, values, offsets, [seed])[0]
    X, feat = _features(family, values)
    centres, labels = _kmeanspp_host(feat, _uniforms(seed, N))
    return _model_from_labels(family, N, X, centres, labels, offsets)
