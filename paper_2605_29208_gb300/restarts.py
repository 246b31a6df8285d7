"""Random restarts and model selection in one batch (the paper's
k-means++ initialisation, Sec. 4.5, and its AIC / BIC / AICc comparison,
Sec. 5.6).

Every restart (and every candidate state count) is its own model of one
multi-model batch: the observations are repeated once per model with that
model's id, so all restarts run in the same kernel launches as independent
problems (the E-step, M-step and Viterbi kernels treat models separately).
Each restart starts from k-means++ with its own seed (all restarts in one
device k-means++ call);
after the fit, one forward pass gives every model's final log-likelihood,
and the library's hmm_information_criteria scores it.
"""
from __future__ import annotations

import numpy as np

from . import Batch, Model, forward_backward, fit, information_criteria
from .initialize import kmeanspp_init_many


def _replicate(values, offsets, R):
    values = np.asarray(values)
    offsets = np.asarray(offsets, np.int64)
    S, TT = len(offsets) - 1, int(offsets[-1])
    vals = np.concatenate([values] * R, axis=0)
    offs = np.concatenate([offsets[:-1] + r * TT for r in range(R)] + [np.array([R * TT], np.int64)])
    mid = np.repeat(np.arange(R, dtype=np.int32), S)
    return vals, offs, mid


def fit_restarts(ctx, family, n_states, values, offsets, n_restarts=8, n_iter=20, seed=0, dim=1):
    """n_restarts fits of an n_states model from k-means++ starts with seeds
    seed, seed + 1, ...; returns (models, loglik per restart, the criteria
    of each restart); the best restart is the one with the largest
    log-likelihood (the criteria order restarts of one state count alike)."""
    R = int(n_restarts)
    inits = kmeanspp_init_many(ctx, family, n_states, values, offsets, [seed + r for r in range(R)])
    vals, offs, mid = _replicate(values, offsets, R)
    model = Model(ctx, inits)
    batch = Batch(vals, offs, mid, dim=dim).make_plan(ctx, model)
    fit(ctx, model, batch, n_iter)
    ll, _, _ = forward_backward(ctx, model, batch, want_gamma=False)
    ll = ll.cpu().numpy()
    S = len(offsets) - 1
    per = np.array([ll[r * S:(r + 1) * S].sum() for r in range(R)])
    n_obs = int(np.asarray(offsets)[-1])
    crit = [information_criteria(family, n_states, float(per[r]), n_obs, dim=dim) for r in range(R)]
    return model.get(), per, crit


def select_states(ctx, family, candidates, values, offsets, n_restarts=4, n_iter=20, seed=0, dim=1,
                  criterion="bic"):
    """For each candidate state count, the best of n_restarts fits; returns
    (best state count, {N: (model, loglik, criteria)}) with the state count
    minimising `criterion` ('aic', 'bic' or 'aicc')."""
    table = {}
    for N in candidates:
        models, ll, crit = fit_restarts(ctx, family, N, values, offsets, n_restarts, n_iter, seed, dim)
        b = int(np.argmax(ll))
        table[N] = (models[b], float(ll[b]), crit[b])
    best = min(table, key=lambda n: table[n][2][criterion])
    return best, table
