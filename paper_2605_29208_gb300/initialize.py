"""Starting parameters for Baum-Welch from the data: seeded k-means++.

The paper names k-means++ initialisation without constants; this module
fixes one reading (it is an input to the fit, not a parity target, and both
the CUDA path and the CPU checker receive its output as their starting
model):

* seeding: the first centre is a uniformly drawn observation, each further
  centre an observation drawn with probability proportional to its squared
  distance to the nearest centre so far (numpy ``default_rng(seed)``);
* Lloyd iterations until no assignment changes or 100 iterations, ties to
  the lowest cluster index, an empty cluster keeps its centre;
* state j's emission from cluster j by moments (Gaussian mean / variance,
  Poisson mean, Gamma and Beta method of moments, ...), variances floored;
* pi uniform, A from the label transitions inside each sequence with one
  added to every count (add-one smoothing), rows normalised.

Host numpy: the initialisation runs once per fit.
"""
from __future__ import annotations

import numpy as np

VAR_FLOOR = 1e-6


def _kmeanspp(X, N, rng, max_iter=100):
    T = X.shape[0]
    centres = np.empty((N, X.shape[1]))
    centres[0] = X[rng.integers(T)]
    d2 = np.sum((X - centres[0]) ** 2, axis=1)
    for j in range(1, N):
        tot = d2.sum()
        i = rng.integers(T) if tot <= 0 else rng.choice(T, p=d2 / tot)
        centres[j] = X[i]
        d2 = np.minimum(d2, np.sum((X - centres[j]) ** 2, axis=1))
    labels = None
    for _ in range(max_iter):
        dist = np.sum((X[:, None, :] - centres[None, :, :]) ** 2, axis=2)
        new = np.argmin(dist, axis=1)            # first minimum: lowest cluster
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for j in range(N):
            sel = labels == j
            if sel.any():
                centres[j] = X[sel].mean(axis=0)
    return centres, labels


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


def kmeanspp_init(family, N, values, offsets, seed=0):
    """Starting model dict for `family` with N states from the packed
    observations (values [total_T] or [total_T, D], offsets [S+1])."""
    rng = np.random.default_rng(seed)
    X = np.asarray(values, np.float64)
    X = X[:, None] if X.ndim == 1 else X
    D = X.shape[1]
    feat = X
    if family == "vonmises":        # cluster angles on the unit circle
        feat = np.stack([np.cos(X[:, 0]), np.sin(X[:, 0])], axis=1)
    centres, labels = _kmeanspp(feat, N, rng)
    # order the states by their first centre coordinate (a stable labelling)
    order = np.argsort(centres[:, 0], kind="stable")
    rank = np.empty(N, np.int64)
    rank[order] = np.arange(N)
    labels = rank[labels]
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
