"""Seeded synthetic workloads shaped like the paper's HMM problems.

This module only draws random numbers: model parameters, hidden state
paths simulated from (pi, A), and observations drawn from each state's
emission distribution (numpy ``default_rng``, PCG64).  It holds none of the
inference or estimation arithmetic, so both the CUDA path and the CPU
checker can consume the same inputs.

Models are plain dicts ``{"family", "pi", "A", "params"}`` with
``params[name]`` an array over states (multivariate families add a
trailing dimension).  Observations are rounded to float32 once, here, and
handed out as float64 copies of those float32 values, so that every
consumer sees bit-identical data.

Parameter names per family (rate parameterisation for the Gamma):
  gauss (mu, sigma2), poisson (lam), gamma (alpha, beta=rate),
  beta (a, b), weibull (k, lam), negbin (r, p), student_t (mu, sigma2, nu),
  vonmises (mu, kappa), diag_gauss (mu[N,D], var[N,D]),
  full_gauss (mu[N,D], cov[N,D,D]), discrete (p[N,K]: symbol probabilities;
  observations are the symbol indices 0..K-1 as floats).
"""
from __future__ import annotations

import numpy as np

MASTER_SEED = 20260603

PARAM_NAMES = {
    "gauss": ("mu", "sigma2"),
    "poisson": ("lam",),
    "gamma": ("alpha", "beta"),
    "beta": ("a", "b"),
    "weibull": ("k", "lam"),
    "negbin": ("r", "p"),
    "student_t": ("mu", "sigma2", "nu"),
    "vonmises": ("mu", "kappa"),
    "diag_gauss": ("mu", "var"),
    "full_gauss": ("mu", "cov"),
    "discrete": ("p",),
    "lognormal": ("mu", "sigma2"),
    "exponential": ("lam",),
    "rayleigh": ("sigma2",),
    "uniform": ("a", "b"),
    "chisq": ("nu",),
    "pareto": ("xm", "alpha"),
}


def make_model(family, pi, A, **params):
    return dict(family=family, pi=np.asarray(pi, np.float64),
                A=np.asarray(A, np.float64),
                params={k: np.asarray(v, np.float64) for k, v in params.items()})


def dirichlet_rows(rng, N, conc):
    A = rng.dirichlet(np.full(N, conc), size=N)
    # rows drawn at a small concentration can contain exact zeros in float64
    # only with vanishing probability; keep them strictly positive anyway
    A = np.maximum(A, 1e-300)
    return A / A.sum(axis=1, keepdims=True)


def random_params(rng, family, N, D=1):
    """Parameter draws used by the benchmark workloads."""
    if family == "gauss":
        return dict(mu=rng.normal(0, 3, N), sigma2=rng.uniform(0.5, 2, N) ** 2)
    if family == "poisson":
        return dict(lam=rng.uniform(0.5, 20, N))
    if family == "gamma":
        return dict(alpha=rng.uniform(1, 10, N), beta=1.0 / rng.uniform(0.5, 3, N))
    if family == "beta":
        return dict(a=rng.uniform(0.8, 8, N), b=rng.uniform(0.8, 8, N))
    if family == "weibull":
        return dict(k=rng.uniform(0.7, 5, N), lam=rng.uniform(0.5, 4, N))
    if family == "negbin":
        return dict(r=rng.uniform(1, 10, N), p=rng.uniform(0.2, 0.8, N))
    if family == "student_t":
        return dict(mu=rng.normal(0, 5, N), sigma2=rng.uniform(0.5, 2, N) ** 2,
                    nu=rng.uniform(2, 30, N))
    if family == "vonmises":
        return dict(mu=rng.uniform(-np.pi, np.pi, N), kappa=rng.uniform(0.5, 20, N))
    if family == "diag_gauss":
        return dict(mu=rng.normal(0, 3, (N, D)), var=rng.uniform(0.2, 2, (N, D)))
    if family == "discrete":      # D = number of symbols; rows Dirichlet(1)
        return dict(p=rng.dirichlet(np.ones(D), size=N))
    if family == "lognormal":     # mu, sigma2 of log y
        return dict(mu=rng.normal(0, 1, N), sigma2=rng.uniform(0.1, 1, N))
    if family == "exponential":
        return dict(lam=rng.uniform(0.2, 5, N))
    if family == "rayleigh":
        return dict(sigma2=rng.uniform(0.2, 4, N))
    if family == "uniform":       # overlapping intervals
        a = rng.uniform(-5, 0, N)
        return dict(a=a, b=a + rng.uniform(1, 6, N))
    if family == "chisq":
        return dict(nu=rng.uniform(1, 10, N))
    if family == "pareto":
        return dict(xm=rng.uniform(0.5, 3, N), alpha=rng.uniform(1.5, 6, N))
    if family == "full_gauss":
        cov = np.empty((N, D, D))
        for j in range(N):
            G = rng.normal(0, np.sqrt(0.1), (10, D))     # Wishart(df=10, I/10)
            cov[j] = G.T @ G + 1e-3 * np.eye(D)
        return dict(mu=rng.normal(0, 2, (N, D)), cov=cov)
    raise ValueError(family)


def component_model(model, d):
    """Component d of an independent-components model dict, as a scalar
    model dict (same pi and A)."""
    pre = f"d{d}."
    return make_model(model["components"][d], model["pi"], model["A"],
                      **{k[len(pre):]: v for k, v in model["params"].items() if k.startswith(pre)})


def indep_model(rng, components, N, conc=1.0):
    """An independent-components model (Sec. 4.5): one scalar family per
    observation dimension, parameters drawn as for that family."""
    params = {}
    for d, f in enumerate(components):
        for k, v in random_params(rng, f, N).items():
            params[f"d{d}.{k}"] = v
    m = make_model("indep", rng.dirichlet(np.ones(N)), dirichlet_rows(rng, N, conc), **params)
    m["components"] = list(components)
    return m


def indep_models(components, N, n_models, seed, conc=1.0):
    rng = np.random.default_rng(seed)
    return [indep_model(rng, components, N, conc) for _ in range(n_models)]


def sample_emissions(rng, model, states):
    """Draw y_t from the emission of state q_t (vectorised over t)."""
    f, p = model["family"], model["params"]
    q = states
    n = len(q)
    if f == "indep":
        return np.stack([sample_emissions(rng, component_model(model, d), q)
                         for d in range(len(model["components"]))], axis=1)
    if f == "discrete":
        cp = np.cumsum(p["p"], axis=1)[q]
        u = rng.random(n)[:, None]
        return np.minimum((u * cp[:, -1:] >= cp).sum(1), cp.shape[1] - 1).astype(np.float64)
    if f == "gauss":
        return p["mu"][q] + np.sqrt(p["sigma2"][q]) * rng.standard_normal(n)
    if f == "poisson":
        return rng.poisson(p["lam"][q]).astype(np.float64)
    if f == "gamma":
        return rng.gamma(p["alpha"][q], 1.0 / p["beta"][q])
    if f == "beta":
        y = rng.beta(p["a"][q], p["b"][q])
        return np.clip(y, 1e-6, 1 - 1e-6)
    if f == "weibull":
        return p["lam"][q] * rng.weibull(p["k"][q])
    if f == "negbin":
        return rng.negative_binomial(p["r"][q], p["p"][q]).astype(np.float64)
    if f == "student_t":
        return p["mu"][q] + np.sqrt(p["sigma2"][q]) * rng.standard_t(p["nu"][q])
    if f == "vonmises":
        return rng.vonmises(p["mu"][q], p["kappa"][q])
    if f == "diag_gauss":
        return p["mu"][q] + np.sqrt(p["var"][q]) * rng.standard_normal((n, p["mu"].shape[1]))
    if f == "lognormal":
        return np.exp(p["mu"][q] + np.sqrt(p["sigma2"][q]) * rng.standard_normal(n))
    if f == "exponential":
        return rng.exponential(1.0 / p["lam"][q])
    if f == "rayleigh":
        return rng.rayleigh(np.sqrt(p["sigma2"][q]))
    if f == "uniform":
        # drawn on the float32 grid inside [a, b] so the rounded value stays in the support
        a, b = p["a"][q], p["b"][q]
        y = np.asarray(a + (b - a) * rng.random(n), np.float32).astype(np.float64)
        lo = np.asarray(a, np.float32).astype(np.float64)
        lo = np.where(lo < a, np.nextafter(lo.astype(np.float32), np.float32(np.inf)).astype(np.float64), lo)
        hi = np.asarray(b, np.float32).astype(np.float64)
        hi = np.where(hi > b, np.nextafter(hi.astype(np.float32), np.float32(-np.inf)).astype(np.float64), hi)
        return np.clip(y, lo, hi)
    if f == "chisq":
        return rng.chisquare(p["nu"][q])
    if f == "pareto":
        # inverse CDF, rounded up onto the float32 grid so y >= xm holds after rounding
        y = p["xm"][q] * (1.0 - rng.random(n)) ** (-1.0 / p["alpha"][q])
        y32 = np.asarray(y, np.float32)
        y32 = np.where(y32.astype(np.float64) < p["xm"][q], np.nextafter(y32, np.float32(np.inf)), y32)
        return y32.astype(np.float64)
    if f == "full_gauss":
        D = p["mu"].shape[1]
        z = rng.standard_normal((n, D))
        L = np.linalg.cholesky(p["cov"])
        return p["mu"][q] + np.einsum("tde,te->td", L[q], z)
    raise ValueError(f)


def simulate_states(rng, pi, A, T):
    """Hidden path q_1..q_T of a Markov chain by inverse-CDF sampling."""
    cpi = np.cumsum(pi)
    cA = np.cumsum(A, axis=1)
    u = rng.random(T)
    q = np.empty(T, dtype=np.int64)
    q[0] = min(np.searchsorted(cpi, u[0] * cpi[-1], side="right"), len(pi) - 1)
    for t in range(1, T):
        row = cA[q[t - 1]]
        q[t] = min(np.searchsorted(row, u[t] * row[-1], side="right"), len(pi) - 1)
    return q


def simulate_many(rng, pi, A, lengths):
    """Paths for many sequences at once: time-major vectorised sampling."""
    S = len(lengths)
    Tmax = int(max(lengths)) if S else 0
    cpi = np.cumsum(pi)
    cA = np.cumsum(A, axis=1)
    N = len(pi)
    Q = np.empty((S, Tmax), dtype=np.int64)
    if Tmax == 0:
        return [Q[s, :0] for s in range(S)]
    u = rng.random((Tmax, S))
    Q[:, 0] = np.minimum((u[0][:, None] * cpi[-1] >= cpi[None, :]).sum(1), N - 1)
    for t in range(1, Tmax):
        rows = cA[Q[:, t - 1]]
        Q[:, t] = np.minimum((u[t][:, None] * rows[:, -1:] >= rows).sum(1), N - 1)
    return [Q[s, :lengths[s]] for s in range(S)]


def to_f32_grid(x):
    """Round observations to float32 once; return float64 copies."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def pack(seqs):
    """Concatenate sequences into the packed ragged layout."""
    lengths = np.array([len(s) for s in seqs], dtype=np.int64)
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    values = np.concatenate(seqs, axis=0) if seqs else np.zeros(0)
    return values, offsets


def _stack_params(models, family):
    names = PARAM_NAMES[family]
    return {n: np.stack([np.asarray(m["params"][n], np.float64) for m in models]) for n in names}


def make_batch_many(seed, models, lengths, model_id):
    """Same output as make_batch for many models at once: the hidden paths of
    all sequences are simulated together (inverse CDF on each sequence's own
    transition rows) and emissions drawn per family with gathered parameters."""
    rng = np.random.default_rng(seed)
    model_id = np.asarray(model_id, dtype=np.int32)
    lengths = np.asarray(lengths, dtype=np.int64)
    S = len(lengths)
    N = len(models[0]["pi"])
    cpi = np.cumsum(np.stack([m["pi"] for m in models]), axis=1)          # [M, N]
    cA = np.cumsum(np.stack([m["A"] for m in models]), axis=2)            # [M, N, N]
    Tmax = int(lengths.max()) if S else 0
    offsets = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    states = np.empty(int(offsets[-1]), dtype=np.int64)
    q = np.minimum((rng.random(S)[:, None] * cpi[model_id, -1:] >= cpi[model_id]).sum(1), N - 1)
    alive = np.arange(S)
    for t in range(Tmax):
        alive = alive[lengths[alive] > t]
        if t == 0:
            cur = q[alive]
        else:
            rows = cA[model_id[alive], cur]
            u = rng.random(len(alive))[:, None]
            cur = np.minimum((u * rows[:, -1:] >= rows).sum(1), N - 1)
        states[offsets[alive] + t] = cur
        # keep `cur` aligned with the next step's survivors
        keep = lengths[alive] > t + 1
        cur = cur[keep]
        alive = alive[keep]
        if len(alive) == 0:
            break
    values = np.empty(len(states))
    seq_of_row = np.repeat(np.arange(S), lengths)
    mrow = model_id[seq_of_row]
    for fam in sorted({m["family"] for m in models}):
        fam_models = [i for i, m in enumerate(models) if m["family"] == fam]
        sel = np.isin(mrow, fam_models)
        if not sel.any():
            continue
        lm = np.searchsorted(np.array(fam_models), mrow[sel])
        P = _stack_params([models[i] for i in fam_models], fam)
        params = {n: v[lm, states[sel]] for n, v in P.items()}
        fake = dict(family=fam, params={n: v for n, v in params.items()})
        values[sel] = sample_emissions(rng, fake, np.arange(sel.sum()))
    return to_f32_grid(values), offsets, model_id


def make_batch(seed, models, lengths, model_id):
    """Simulate one sequence per entry of ``lengths`` from
    ``models[model_id[s]]``; returns (values, offsets, model_id)."""
    rng = np.random.default_rng(seed)
    model_id = np.asarray(model_id, dtype=np.int32)
    lengths = np.asarray(lengths, dtype=np.int64)
    seqs = [None] * len(lengths)
    for m, model in enumerate(models):
        idx = np.nonzero(model_id == m)[0]
        if len(idx) == 0:
            continue
        paths = simulate_many(rng, model["pi"], model["A"], lengths[idx])
        for s, q in zip(idx, paths):
            seqs[s] = to_f32_grid(sample_emissions(rng, model, q))
    values, offsets = pack(seqs)
    return values, offsets, model_id


def perturb(rng, model, frac=0.2):
    """EM start: parameters scaled by U[1-frac, 1+frac], A <- A/2 + 1/(2N),
    pi uniform."""
    N = len(model["pi"])
    if model["family"] == "indep":
        params = {}
        for d in range(len(model["components"])):
            for k, v in perturb(rng, component_model(model, d), frac)["params"].items():
                params[f"d{d}.{k}"] = v
        m = make_model("indep", np.full(N, 1.0 / N), 0.5 * model["A"] + 0.5 / N, **params)
        m["components"] = list(model["components"])
        return m
    params = {}
    for k, v in model["params"].items():
        if model["family"] in ("vonmises",) and k == "mu":
            params[k] = v + rng.uniform(-0.3, 0.3, v.shape)
        elif model["family"] in ("gauss", "student_t", "diag_gauss", "full_gauss") and k == "mu":
            params[k] = v + rng.uniform(-0.3, 0.3, v.shape)
        elif model["family"] == "discrete":
            q = v * rng.uniform(1 - frac, 1 + frac, v.shape)
            params[k] = q / q.sum(axis=1, keepdims=True)
        elif model["family"] == "uniform":
            # widened, so that every observation stays inside its state's support
            w = (model["params"]["b"] - model["params"]["a"]) * rng.uniform(0, frac, v.shape)
            params[k] = v - w if k == "a" else v + w
        elif model["family"] == "pareto" and k == "xm":
            params[k] = v * rng.uniform(1 - frac, 1, v.shape)   # lowered: the support only grows
        elif k == "p":
            params[k] = np.clip(v * rng.uniform(1 - frac, 1 + frac, v.shape), 0.02, 0.98)
        elif k == "cov":
            params[k] = v * rng.uniform(1 - frac, 1 + frac, (v.shape[0], 1, 1))
        else:
            params[k] = v * rng.uniform(1 - frac, 1 + frac, v.shape)
    return make_model(model["family"], np.full(N, 1.0 / N),
                      0.5 * model["A"] + 0.5 / N, **params)


# --------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped benchmark configurations)
# --------------------------------------------------------------------------
def tiny_gauss(seed=MASTER_SEED):
    """2-state univariate Gaussian, means (-1, +1), sd 1,
    A = [[.9,.1],[.1,.9]], pi uniform, one sequence of T = 1000."""
    truth = make_model("gauss", [0.5, 0.5], [[0.9, 0.1], [0.1, 0.9]],
                       mu=[-1.0, 1.0], sigma2=[1.0, 1.0])
    values, offsets, mid = make_batch(seed, [truth], [1000], [0])
    return truth, values, offsets, mid


def scale_workload(family, n_seq=4096, T=2000, N=16, seed=MASTER_SEED + 1):
    """N = 16 states, 4096 sequences of T = 2000, one shared model with
    Dirichlet(1) transition rows, pi uniform; Gamma (shape ~ U[1,10],
    scale ~ U[0.5,3]) or Student-t (nu ~ U[2,30], loc ~ N(0,5),
    scale ~ U[0.5,2]) emissions.  Returns (truth, init, values, offsets,
    model_id); the EM start is the truth perturbed."""
    rng = np.random.default_rng(seed)
    truth = make_model(family, np.full(N, 1.0 / N), dirichlet_rows(rng, N, 1.0),
                       **random_params(rng, family, N))
    init = perturb(rng, truth)
    values, offsets, mid = make_batch(seed + 100, [truth], [T] * n_seq, [0] * n_seq)
    return truth, init, values, offsets, mid


BATCH_FAMILIES = ("gauss", "poisson", "negbin", "vonmises")


def batching_workload(n_seq=100_000, n_models=1024, N=8, seed=MASTER_SEED + 2,
                      median=500, sigma=1.0, tmin=50, tmax=20000, families=BATCH_FAMILIES):
    """Ragged batch: lengths round(lognormal(log median, sigma)) clipped to
    [tmin, tmax]; n_models models, each with one family drawn uniformly from
    Gaussian / Poisson / negative binomial / von Mises for all its states;
    sequences assigned to models uniformly."""
    rng = np.random.default_rng(seed)
    lengths = np.clip(np.round(rng.lognormal(np.log(median), sigma, n_seq)),
                      tmin, tmax).astype(np.int64)
    fams = rng.integers(0, len(families), n_models)
    truths, inits = [], []
    for m in range(n_models):
        fam = families[fams[m]]
        t = make_model(fam, np.full(N, 1.0 / N), dirichlet_rows(rng, N, 1.0),
                       **random_params(rng, fam, N))
        truths.append(t)
        inits.append(perturb(rng, t))
    model_id = rng.integers(0, n_models, n_seq).astype(np.int32)
    values, offsets, mid = make_batch_many(seed + 100, truths, lengths, model_id)
    return truths, inits, values, offsets, mid


def large_state_workload(n_seq=1024, T=4096, N=512, D=32, seed=MASTER_SEED + 3):
    """N = 512 states with Dirichlet(0.1) transition rows, diagonal
    Gaussian emissions of dimension D = 32 (means N(0,3), variances
    U[0.2,2]), n_seq sequences of length T, one shared model."""
    rng = np.random.default_rng(seed)
    truth = make_model("diag_gauss", np.full(N, 1.0 / N), dirichlet_rows(rng, N, 0.1),
                       **random_params(rng, "diag_gauss", N, D))
    init = perturb(rng, truth)
    values, offsets, mid = make_batch(seed + 100, [truth], [T] * n_seq, [0] * n_seq)
    return truth, init, values, offsets, mid


def small_models(family, N, n_models, seed, conc=1.0, D=1):
    rng = np.random.default_rng(seed)
    return [make_model(family, rng.dirichlet(np.ones(N)), dirichlet_rows(rng, N, conc),
                       **random_params(rng, family, N, D)) for _ in range(n_models)]


def serving_workload(n_req=1000, rate=2000.0, t_min=100, t_max=100000, seed=MASTER_SEED + 5):
    """Request stream for the server: Poisson arrivals at `rate` per second;
    kind decode / posterior / fit (10 iterations) with probabilities 0.5 / 0.3
    / 0.2; N uniform in {4, 16, 64, 256}; T log-uniform in [t_min, t_max];
    emissions full-covariance Gaussian D = 8 (Wishart covariances) or Gamma,
    half each; every request has its own model (fit requests start from a
    perturbed copy).  Returns a list of dicts (arrival_s, kind, model,
    values, n_iter) in arrival order."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    kinds = rng.choice(["decode", "posterior", "fit"], size=n_req, p=[0.5, 0.3, 0.2])
    Ns = rng.choice([4, 16, 64, 256], size=n_req)
    Ts = np.round(np.exp(rng.uniform(np.log(t_min), np.log(t_max), n_req))).astype(np.int64)
    fams = rng.choice(["full_gauss", "gamma"], size=n_req)
    reqs = [None] * n_req
    # hidden paths: all requests with the same N at once (time-major, vectorised)
    for N in (4, 16, 64, 256):
        idx = np.nonzero(Ns == N)[0]
        if len(idx) == 0:
            continue
        models = []
        for i in idx:
            D = 8 if fams[i] == "full_gauss" else 1
            models.append(make_model(fams[i], np.full(N, 1.0 / N), dirichlet_rows(rng, N, 1.0),
                                     **random_params(rng, fams[i], N, D)))
        lengths = Ts[idx]
        cA = np.cumsum(np.stack([m["A"] for m in models]), axis=2)
        S = len(idx)
        offsets = np.zeros(S + 1, np.int64)
        np.cumsum(lengths, out=offsets[1:])
        states = np.empty(int(offsets[-1]), np.int64)
        cur = rng.integers(0, N, S)
        alive = np.arange(S)
        for t in range(int(lengths.max())):
            alive_now = alive[lengths[alive] > t]
            if t > 0:
                rows = cA[alive_now, cur[alive_now]]
                u = rng.random(len(alive_now))[:, None]
                cur[alive_now] = np.minimum((u * rows[:, -1:] >= rows).sum(1), N - 1)
            states[offsets[alive_now] + t] = cur[alive_now]
            alive = alive_now
        for k, i in enumerate(idx):
            q = states[offsets[k]:offsets[k + 1]]
            y = sample_emissions(rng, models[k], q)
            y = np.asarray(y, np.float32)
            init = perturb(rng, models[k]) if kinds[i] == "fit" else models[k]
            reqs[i] = dict(arrival_s=float(arrivals[i]), kind=str(kinds[i]), model=init, values=y,
                           n_iter=10 if kinds[i] == "fit" else 0)
    return reqs
