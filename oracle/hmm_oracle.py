"""Plain, slow FP64 CPU oracle for the HMM hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this file;
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and ``--impl reference`` arm) may import or run it.  It shares no
code with the CUDA path.

Everything here is the plain definition from the paper (libhmm,
arXiv 2605.29208), evaluated in float64 with numpy/scipy library primitives
(``logaddexp``-free: the log-sum-exp is written out as the paper defines it).
Citations name the paper's section and equation numbers:

  Sec. 3.2  log-space forward-backward, Eq. 1 (init) and Eq. 2 (recursion);
            the backward pass and smoothed probabilities "analogously".
  Sec. 3.1  notation: gamma_t(j), xi_t(i,j).
  Sec. 3.3  Viterbi, Eq. 3-4 with the backpointer psi_t(j).
  Sec. 3.4  posterior decoding q_t = argmax_j gamma_t(j).
  Sec. 4    weighted M-step, Eq. 5 (N_j, ybar_j) and Eq. 6 (argmax).
  Sec. 4.1  closed forms (Gaussian, Poisson, von Mises mean direction).
  Sec. 4.2  Newton-Raphson: Gamma (Eq. 7-8), Beta (Eq. 9-10), Weibull
            (Eq. 11), von Mises kappa (Eq. 12), negative binomial (text).
  Sec. 4.3  ECME for Student-t: Eq. 13 (scale mixture), Eq. 14 (u-tilde),
            Eq. 15-16 (CM-step 1), Eq. 17-19 (CM-step 2 for nu).
  Sec. 4.4  state-collapse guard (N_j < 1e-8 keeps the parameters).
  Sec. 4.5  diagonal Gaussian (Eq. 20-21), full covariance (Eq. 22-24).
  Sec. 4    closed forms of the further scalar families: log-normal,
            exponential, Rayleigh, uniform, discrete; Sec. 4.2 chi-squared
            (Gamma with beta = 1/2, one parameter) and Pareto (min, then a
            closed-form shape).

Where the paper is silent the readings used are listed in the module
constants and functions below (transition/initial M-step, tie breaks,
support of each family, Newton stopping rule, negative-binomial score,
the Student-t nu equation, Weibull seed).

Parity status: every function here is pinned by the not-gpu tests in
``tests/test_oracle_*.py`` (brute-force path enumeration, invariants,
closed forms, scipy.stats fits, score equations).  None is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import linalg as sla
from scipy import special as sp

# --------------------------------------------------------------------------
# Readings where the paper is silent (also listed in the design notes)
# --------------------------------------------------------------------------
COLLAPSE_EPS = 1e-8          # Sec. 4.4: skip the M-step for state j if N_j < eps
TIKHONOV_EPS = 1e-6          # Sec. 4.5: Sigma + eps I for the full covariance
NEWTON_TOL = 1e-10           # |delta| <= tol * max(1, |theta|) stops Newton
NEWTON_MAXIT = 50
NU_TOL = 1e-6                # Sec. 4.3: |d nu| < 1e-6 stops the nu Newton
NU_MIN, NU_MAX = 0.5, 1e4    # reading: nu kept in [0.5, 1e4]
NEGBIN_RMAX = 1e6            # reading: no finite MLE when var <= mean
KAPPA_MAX = 1e6              # reading: R -> 1 gives kappa -> inf
VAR_RESOLUTION = 1e-6        # reading 14: a variance below this fraction of the
                             # weighted mean square deviation from the current
                             # location counts as zero (an undefined update)

FAMILIES = ("gauss", "poisson", "gamma", "beta", "weibull", "negbin",
            "student_t", "vonmises", "diag_gauss", "full_gauss", "discrete",
            "lognormal", "exponential", "rayleigh", "uniform", "chisq", "pareto",
            "indep")


@dataclass
class Model:
    """lambda = (pi, A, B) of Sec. 3.1 with the emission family of every
    state equal to ``family`` and parameters ``params[name][j]``."""
    family: str
    pi: np.ndarray            # [N]
    A: np.ndarray             # [N, N] row-stochastic
    params: dict = field(default_factory=dict)
    # family "indep" (Sec. 4.5, independent components): the scalar family
    # of each observation dimension; parameters are named "d<k>.<name>"
    components: tuple = ()

    @property
    def n_states(self) -> int:
        return self.A.shape[0]

    def copy(self) -> "Model":
        return Model(self.family, self.pi.copy(), self.A.copy(),
                     {k: np.array(v, dtype=np.float64, copy=True)
                      for k, v in self.params.items()}, tuple(self.components))


def component_model(model: Model, d: int) -> Model:
    """The scalar model of dimension d of an independent-components model
    (same pi and A; the parameters of component d)."""
    pre = f"d{d}."
    return Model(model.components[d], model.pi, model.A,
                 {k[len(pre):]: v for k, v in model.params.items() if k.startswith(pre)})


# --------------------------------------------------------------------------
# log-sum-exp exactly as Sec. 3.2 defines it: max + log sum exp(x - max)
# --------------------------------------------------------------------------
def lse(x: np.ndarray, axis: int) -> np.ndarray:
    m = np.max(x, axis=axis, keepdims=True)
    finite = np.isfinite(m)
    m0 = np.where(finite, m, 0.0)
    with np.errstate(divide="ignore"):
        out = m0 + np.log(np.sum(np.exp(x - m0), axis=axis, keepdims=True))
    out = np.where(finite, out, m)          # all -inf stays -inf
    return np.squeeze(out, axis=axis)


# --------------------------------------------------------------------------
# Emission log-densities log b_j(y_t) -> [T, N]
# --------------------------------------------------------------------------
def _is_count(y):
    return (y >= 0) & (np.floor(y) == y)


def emission_logpdf(model: Model, y: np.ndarray) -> np.ndarray:
    """log b_j(y_t) for every t and state j (densities of Sec. 4.1-4.5).

    Scalar families take y of shape [T]; the multivariate ones [T, D].
    Observations outside a family's support give -inf (reading).
    """
    f, p = model.family, model.params
    y = np.asarray(y, dtype=np.float64)
    if f == "indep":            # Sec. 4.5: b_j(y) = prod_d phi_d(y_d)
        y = y.reshape(len(y), -1)
        return sum(emission_logpdf(component_model(model, d), y[:, d]) for d in range(len(model.components)))
    with np.errstate(divide="ignore", invalid="ignore"):
        if f == "gauss":        # Sec. 4.1, N(mu, sigma^2)
            mu, s2 = p["mu"], p["sigma2"]
            yy = y[:, None]
            return -0.5 * np.log(2 * np.pi * s2) - (yy - mu) ** 2 / (2 * s2)
        if f == "poisson":      # Sec. 4.1
            lam = p["lam"]
            yy = y[:, None]
            out = yy * np.log(lam) - lam - sp.gammaln(yy + 1)
            return np.where(_is_count(yy), out, -np.inf)
        if f == "gamma":        # Sec. 4.2, rate parameterisation (beta = rate)
            a, b = p["alpha"], p["beta"]
            yy = y[:, None]
            out = a * np.log(b) + (a - 1) * np.log(yy) - b * yy - sp.gammaln(a)
            return np.where(yy > 0, out, -np.inf)
        if f == "beta":         # Sec. 4.2
            a, b = p["a"], p["b"]
            yy = y[:, None]
            out = (a - 1) * np.log(yy) + (b - 1) * np.log1p(-yy) - sp.betaln(a, b)
            return np.where((yy > 0) & (yy < 1), out, -np.inf)
        if f == "weibull":      # Sec. 4.2, shape k, scale lambda
            k, lam = p["k"], p["lam"]
            yy = y[:, None]
            out = (np.log(k) - k * np.log(lam) + (k - 1) * np.log(yy)
                   - (yy / lam) ** k)
            return np.where(yy > 0, out, -np.inf)
        if f == "negbin":       # Sec. 4.2, p = r / (r + mean)
            r, pp = p["r"], p["p"]
            yy = y[:, None]
            out = (sp.gammaln(yy + r) - sp.gammaln(r) - sp.gammaln(yy + 1)
                   + r * np.log(pp) + yy * np.log1p(-pp))
            return np.where(_is_count(yy), out, -np.inf)
        if f == "student_t":    # Sec. 4.3, location-scale t
            mu, s2, nu = p["mu"], p["sigma2"], p["nu"]
            yy = y[:, None]
            return (sp.gammaln((nu + 1) / 2) - sp.gammaln(nu / 2)
                    - 0.5 * np.log(nu * np.pi * s2)
                    - (nu + 1) / 2 * np.log1p((yy - mu) ** 2 / (nu * s2)))
        if f == "vonmises":     # Sec. 4.1-4.2, log(2 pi I0(k)) = log 2pi + log i0e(k) + k
            mu, kap = p["mu"], p["kappa"]
            yy = y[:, None]
            return (kap * np.cos(yy - mu) - np.log(2 * np.pi)
                    - (np.log(sp.i0e(kap)) + kap))
        if f == "diag_gauss":   # Sec. 4.5, Eq. 20
            mu, var = p["mu"], p["var"]          # [N, D]
            d = y[:, None, :] - mu[None]
            return np.sum(-0.5 * np.log(2 * np.pi * var)[None]
                          - d ** 2 / (2 * var[None]), axis=2)
        if f == "discrete":     # Sec. 4, "Discrete (categorical)": b_j(k) = p_jk
            pk = p["p"]                          # [N, K]
            K = pk.shape[1]
            ok = _is_count(y) & (y < K)
            idx = np.where(ok, y, 0).astype(np.int64)
            out = np.log(pk[:, idx]).T           # [T, N]
            return np.where(ok[:, None], out, -np.inf)
        if f == "lognormal":    # Sec. 4.1 "Log-normal": a Gaussian on log y, y > 0
            mu, s2 = p["mu"], p["sigma2"]
            yy = y[:, None]
            ly = np.log(np.where(yy > 0, yy, 1.0))
            out = -ly - 0.5 * np.log(2 * np.pi * s2) - (ly - mu) ** 2 / (2 * s2)
            return np.where(yy > 0, out, -np.inf)
        if f == "exponential":  # Sec. 4.1 "Exponential": rate lambda, y >= 0
            lam = p["lam"]
            yy = y[:, None]
            out = np.log(lam) - lam * yy
            return np.where(yy >= 0, out, -np.inf)
        if f == "rayleigh":     # Sec. 4.1 "Rayleigh": y / s2 exp(-y^2 / (2 s2)), y >= 0
            s2 = p["sigma2"]
            yy = y[:, None]
            out = np.log(yy) - np.log(s2) - yy ** 2 / (2 * s2)
            return np.where(yy >= 0, out, -np.inf)
        if f == "uniform":      # Sec. 4.1 "Uniform": 1 / (b - a) on the closed interval [a, b]
            a, b = p["a"], p["b"]
            yy = y[:, None]
            out = -np.log(b - a) + 0 * yy
            return np.where((yy >= a) & (yy <= b), out, -np.inf)
        if f == "chisq":        # Sec. 4.2 "Chi-squared": Gamma(nu / 2, rate 1/2), y > 0
            nu = p["nu"]
            yy = y[:, None]
            ly = np.log(np.where(yy > 0, yy, 1.0))
            out = (nu / 2 - 1) * ly - yy / 2 - nu / 2 * np.log(2.0) - sp.gammaln(nu / 2)
            return np.where(yy > 0, out, -np.inf)
        if f == "pareto":       # Sec. 4.2 "Pareto": alpha xm^alpha / y^(alpha+1), y >= xm
            xm, al = p["xm"], p["alpha"]
            yy = y[:, None]
            ly = np.log(np.where(yy > 0, yy, 1.0))
            out = np.log(al) + al * np.log(xm) - (al + 1) * ly
            return np.where(yy >= xm, out, -np.inf)
        if f == "full_gauss":   # Sec. 4.5, Eq. 22 through the Cholesky factor
            mu, cov = p["mu"], p["cov"]          # [N, D], [N, D, D]
            T, D = y.shape
            out = np.empty((T, mu.shape[0]))
            for j in range(mu.shape[0]):
                L = np.linalg.cholesky(cov[j])
                z = sla.solve_triangular(L, (y - mu[j]).T, lower=True)
                out[:, j] = (-0.5 * D * np.log(2 * np.pi)
                             - np.sum(np.log(np.diag(L)))
                             - 0.5 * np.sum(z * z, axis=0))
            return out
    raise ValueError(f"unknown family {f!r}")


# --------------------------------------------------------------------------
# Forward / backward in log space (Sec. 3.2)
# --------------------------------------------------------------------------
def forward_log(logpi, logA, logb):
    """alpha-hat_t(j) by Eq. 1 and Eq. 2.  logb: [T, N]."""
    T, N = logb.shape
    alpha = np.empty((T, N))
    alpha[0] = logpi + logb[0]                                   # Eq. 1
    for t in range(1, T):                                        # Eq. 2
        alpha[t] = lse(alpha[t - 1][:, None] + logA, axis=0) + logb[t]
    return alpha


def backward_log(logA, logb):
    """beta-hat_t(i) = log P(y_{t+1..T} | q_t = i): beta-hat_T = 0 and
    beta-hat_t(i) = lse_j[log a_ij + log b_j(y_{t+1}) + beta-hat_{t+1}(j)]
    (the 'analogous' backward recursion of Sec. 3.2)."""
    T, N = logb.shape
    beta = np.empty((T, N))
    beta[T - 1] = 0.0
    for t in range(T - 2, -1, -1):
        beta[t] = lse(logA + (logb[t + 1] + beta[t + 1])[None, :], axis=1)
    return beta


def forward_backward_logb(logpi, logA, logb):
    """logL, gamma_t(j), sum_t xi_t(i,j) (Sec. 3.1 definitions) from a
    log-emission table."""
    alpha = forward_log(logpi, logA, logb)
    beta = backward_log(logA, logb)
    logL = float(lse(alpha[-1], axis=0))
    gamma = np.exp(alpha + beta - logL)
    T, N = logb.shape
    xi_sum = np.zeros((N, N))
    for t in range(T - 1):
        xi_sum += np.exp(alpha[t][:, None] + logA
                         + (logb[t + 1] + beta[t + 1])[None, :] - logL)
    return dict(logL=logL, gamma=gamma, xi_sum=xi_sum, alpha=alpha, beta=beta)


def _logs(model: Model):
    with np.errstate(divide="ignore"):
        return np.log(model.pi), np.log(model.A)


def forward_backward(model: Model, y):
    logpi, logA = _logs(model)
    return forward_backward_logb(logpi, logA, emission_logpdf(model, y))


def posterior_decode(gamma):
    """Sec. 3.4: argmax_j gamma_t(j); ties go to the lowest j (reading)."""
    return np.argmax(gamma, axis=1).astype(np.int32)


# --------------------------------------------------------------------------
# Viterbi (Sec. 3.3)
# --------------------------------------------------------------------------
def viterbi_logb(logpi, logA, logb):
    """Max-plus recursion of Eq. 3-4 in FP64 with backpointers.

    Ties (reading): scanning i upward with a strict '>' keeps the lowest
    predecessor index; the final state is the lowest index attaining the
    maximum.  Returns (path [T] int32, score float)."""
    T, N = logb.shape
    delta = logpi + logb[0]
    psi = np.zeros((T, N), dtype=np.int32)
    for t in range(1, T):
        cand = delta[:, None] + logA                   # [i, j]
        psi[t] = np.argmax(cand, axis=0)               # first max = lowest i
        delta = cand[psi[t], np.arange(N)] + logb[t]
    q = np.empty(T, dtype=np.int32)
    q[T - 1] = int(np.argmax(delta))
    for t in range(T - 1, 0, -1):
        q[t - 1] = psi[t, q[t]]
    return q, float(delta[q[T - 1]])


def viterbi(model: Model, y):
    logpi, logA = _logs(model)
    return viterbi_logb(logpi, logA, emission_logpdf(model, y))


def viterbi_gaps(logpi, logA, logb):
    """FP64 best-minus-second-best margins of every Viterbi decision, used
    to excuse path differences at near-ties.  Returns (path, score,
    step_gap [T, N], final_gap) where step_gap[t, j] is the margin of the
    predecessor choice psi_t(j)."""
    T, N = logb.shape
    delta = logpi + logb[0]
    psi = np.zeros((T, N), dtype=np.int32)
    gap = np.full((T, N), np.inf)
    for t in range(1, T):
        cand = delta[:, None] + logA
        psi[t] = np.argmax(cand, axis=0)
        srt = np.sort(cand, axis=0)
        if N > 1:
            gap[t] = srt[-1] - srt[-2]
        delta = cand[psi[t], np.arange(N)] + logb[t]
    q = np.empty(T, dtype=np.int32)
    q[T - 1] = int(np.argmax(delta))
    fs = np.sort(delta)
    final_gap = float(fs[-1] - fs[-2]) if N > 1 else np.inf
    for t in range(T - 1, 0, -1):
        q[t - 1] = psi[t, q[t]]
    return q, float(delta[q[T - 1]]), gap, final_gap


def viterbi_fp32(logpi32, logA32, logb32):
    """Viterbi in float32 with a fixed operation order, for bit-exact
    comparison of decoded paths (reading of Sec. 3.3 for a single-precision
    device).  Only IEEE additions, subtractions and comparisons occur:

      delta_1(j) = logpi(j) + logb_1(j)
      for t >= 2, every j: scan i = 0..N-1 upward,
          c = delta_{t-1}(i) + logA(i, j); keep c if c > best (strict)
      delta_t(j) = best + logb_t(j)
      after every step m_t = max_j delta_t(j) and, if m_t is finite,
      delta_t(j) <- delta_t(j) - m_t, with m_t added to an FP64 score.
    The final state is the lowest j with delta_T(j) == max_j delta_T(j).
    Returns (path int32 [T], score float64)."""
    f32 = np.float32
    logpi32 = np.asarray(logpi32, dtype=f32)
    logA32 = np.asarray(logA32, dtype=f32)
    logb32 = np.asarray(logb32, dtype=f32)
    T, N = logb32.shape
    if T == 0:                      # an empty sequence: empty path, log 1 = 0
        return np.zeros(0, np.int32), 0.0
    psi = np.zeros((T, N), dtype=np.int32)
    d = (logpi32 + logb32[0]).astype(f32)
    off = 0.0
    m = d.max()
    if np.isfinite(m):
        d = (d - m).astype(f32)
        off += float(m)
    for t in range(1, T):
        # c(i, j) = delta_{t-1}(i) + logA(i, j) in float32; the first
        # maximum over i (lowest index) is what a strict '>' scan keeps.
        cand = (d[:, None] + logA32).astype(f32)
        psi[t] = np.argmax(cand, axis=0)
        best = cand[psi[t], np.arange(N)]
        nd = (best + logb32[t]).astype(f32)
        m = nd.max()
        if np.isfinite(m):
            nd = (nd - m).astype(f32)
            off += float(m)
        d = nd
    q = np.empty(T, dtype=np.int32)
    q[T - 1] = int(np.argmax(d))
    score = off + float(d[q[T - 1]])
    for t in range(T - 1, 0, -1):
        q[t - 1] = psi[t, q[t]]
    return q, score


def _shift32(v, off):
    """Subtract the float32 maximum when it is finite; the shift goes to the
    float64 offset."""
    m = v.max()
    if np.isfinite(m):
        return (v - m).astype(np.float32), off + float(m)
    return v, off


def viterbi_fp32_mitm(logpi32, logA32, logb32):
    """Viterbi decoded from both ends in float32 (the reading of Sec. 3.3,
    Eq. 3-4, used by the device for small state counts), with a fixed
    operation order so that decoded paths can be compared bit for bit.

    With h = floor(T/2):
      forward, t = 0..h: delta_0(j) = logpi(j) + logb_0(j); for t >= 1
          c(i, j) = delta_{t-1}(i) + logA(i, j), psi_t(j) = lowest i
          attaining max_i c(i, j), delta_t(j) = c(psi_t(j), j) + logb_t(j);
      backward, t = T-1..h: beta_{T-1}(i) = 0; for t < T-1
          v(j) = beta_{t+1}(j) + logb_{t+1}(j),
          c(i, j) = v(j) + logA(i, j), phi_t(i) = lowest j attaining
          max_j c(i, j), beta_t(i) = c(i, phi_t(i));
      after every step of either chain its maximum, when finite, is
      subtracted and added to that chain's float64 offset;
      meeting point: q_h = lowest j attaining max_j delta_h(j) + beta_h(j);
      q_{t-1} = psi_t(q_t) for t = h..1, q_{t+1} = phi_t(q_t) for t = h..T-2.
    Every operation on the scores is a float32 addition, subtraction or
    comparison.  The score is max_j (delta_h(j) + beta_h(j)) plus both
    offsets.  Returns (path int32 [T], score float64)."""
    f32 = np.float32
    logpi32 = np.asarray(logpi32, dtype=f32)
    logA32 = np.asarray(logA32, dtype=f32)
    logb32 = np.asarray(logb32, dtype=f32)
    T, N = logb32.shape
    if T == 0:
        return np.zeros(0, np.int32), 0.0
    h = T // 2
    cols = np.arange(N)
    psi = np.zeros((T, N), dtype=np.int32)
    d, doff = _shift32((logpi32 + logb32[0]).astype(f32), 0.0)
    for t in range(1, h + 1):
        cand = (d[:, None] + logA32).astype(f32)        # [i, j]
        psi[t] = np.argmax(cand, axis=0)                 # lowest i at ties
        d, doff = _shift32((cand[psi[t], cols] + logb32[t]).astype(f32), doff)
    phi = np.zeros((T, N), dtype=np.int32)
    b, boff = _shift32(np.zeros(N, dtype=f32), 0.0)
    for t in range(T - 2, h - 1, -1):
        v = (b + logb32[t + 1]).astype(f32)
        cand = (v[None, :] + logA32).astype(f32)        # [i, j]
        phi[t] = np.argmax(cand, axis=1)                 # lowest j at ties
        b, boff = _shift32(cand[cols, phi[t]].astype(f32), boff)
    c = (d + b).astype(f32)
    q = np.empty(T, dtype=np.int32)
    q[h] = int(np.argmax(c))
    for t in range(h, 0, -1):
        q[t - 1] = psi[t, q[t]]
    for t in range(h, T - 1):
        q[t + 1] = phi[t, q[t]]
    return q, doff + boff + float(c[q[h]])


def path_logprob(logpi, logA, logb, path):
    """log P(q, y) of one state path (the product whose maximum Eq. 3
    takes): log pi_{q_1} + sum_t log a_{q_{t-1} q_t} + sum_t log b_{q_t}(y_t),
    in float64."""
    path = np.asarray(path, dtype=np.int64)
    T = len(path)
    if T == 0:
        return 0.0
    lp = float(logpi[path[0]])
    lp += float(np.sum(logA[path[:-1], path[1:]]))
    lp += float(np.sum(logb[np.arange(T), path]))
    return lp


# --------------------------------------------------------------------------
# Special functions used by the M-steps (library routines)
# --------------------------------------------------------------------------
def digamma(x):
    return sp.digamma(x)


def trigamma(x):
    return sp.polygamma(1, x)


def bessel_ratio(kappa):
    """A(kappa) = I1(kappa) / I0(kappa) (Sec. 4.2), through the
    exponentially scaled Bessel functions so that large kappa is safe."""
    return sp.i1e(kappa) / sp.i0e(kappa)


# --------------------------------------------------------------------------
# Weighted M-steps for one state (Sec. 4), w = gamma_t(j) over the
# concatenated sequences of one model, y the matching observations.
# --------------------------------------------------------------------------
def _positive_step(x, step):
    """Newton iterate x - step with the step halved until it is positive, at
    most 64 times (reading: the paper's 'step halving' bound); NaN if that
    fails, which makes the update undefined (see valid_update)."""
    for _ in range(64):
        new = x - step
        if new > 0 and np.isfinite(new):
            return new
        step *= 0.5
    return np.nan


def _newton_done(old, new):
    return abs(new - old) <= NEWTON_TOL * max(1.0, abs(old))


def mstep_gauss(w, y, cur):
    """Sec. 4.1: mu = ybar, sigma^2 = N^-1 sum w (y - mu)^2 (two-pass)."""
    Nj = w.sum()
    mu = np.sum(w * y) / Nj
    s2 = np.sum(w * (y - mu) ** 2) / Nj
    if s2 <= VAR_RESOLUTION * np.sum(w * (y - cur.get("mu", mu)) ** 2) / Nj:
        s2 = 0.0                    # e.g. one observation: undefined, theta_j kept
    return dict(mu=mu, sigma2=s2)


def mstep_poisson(w, y, cur):
    """Sec. 4.1: lambda = ybar."""
    return dict(lam=np.sum(w * y) / w.sum())


def mstep_gamma(w, y, cur):
    """Sec. 4.2, Eq. 7-8: Newton on the shape from the MOM seed
    ybar^2 / sigma^2, rate = shape / ybar.  (The N_j factors of Eq. 7 and
    Eq. 8 cancel in the update.)"""
    Nj = w.sum()
    ybar = np.sum(w * y) / Nj
    mlog = np.sum(w * np.log(y)) / Nj
    c = np.log(ybar) - mlog
    var = np.sum(w * (y - ybar) ** 2) / Nj
    a = ybar * ybar / var
    iters = 0
    for iters in range(1, NEWTON_MAXIT + 1):
        s = np.log(a) - digamma(a) - c
        ds = 1.0 / a - trigamma(a)
        new = _positive_step(a, s / ds)
        done = _newton_done(a, new)
        a = new
        if done:
            break
    return dict(alpha=a, beta=a / ybar, _iters=iters)


def mstep_beta(w, y, cur):
    """Sec. 4.2, Eq. 9-10: joint Newton on
    psi(a) - psi(a+b) = mean log y, psi(b) - psi(a+b) = mean log(1-y)
    with the trigamma Jacobian, from the MOM seeds of the text.
    Reading: if the MOM seed is not positive, start from (1, 1)."""
    Nj = w.sum()
    ybar = np.sum(w * y) / Nj
    var = np.sum(w * (y - ybar) ** 2) / Nj
    m1 = np.sum(w * np.log(y)) / Nj
    m2 = np.sum(w * np.log1p(-y)) / Nj
    k = ybar * (1 - ybar) / var - 1
    a, b = (ybar * k, (1 - ybar) * k) if k > 0 else (1.0, 1.0)
    iters = 0
    for iters in range(1, NEWTON_MAXIT + 1):
        pab = digamma(a + b)
        F = np.array([digamma(a) - pab - m1, digamma(b) - pab - m2])
        tab = trigamma(a + b)
        J = np.array([[trigamma(a) - tab, -tab], [-tab, trigamma(b) - tab]])
        step = np.linalg.solve(J, F)
        na, nb = a - step[0], b - step[1]
        for _ in range(64):
            if na > 0 and nb > 0:
                break
            step *= 0.5
            na, nb = a - step[0], b - step[1]
        if not (na > 0 and nb > 0):
            na = nb = np.nan
        done = _newton_done(a, na) and _newton_done(b, nb)
        a, b = na, nb
        if done:
            break
    return dict(a=a, b=b, _iters=iters)


def mstep_weibull(w, y, cur):
    """Sec. 4.2, Eq. 11: Newton on
    f(k) = 1/k + mean log y - sum w y^k log y / sum w y^k, with
    f'(k) = -1/k^2 - (S2 S0 - S1^2) / S0^2, S_r = sum w y^k (log y)^r;
    scale = (N^-1 sum w y^k)^(1/k).  Reading for the 'MOM seed': log Y of a
    Weibull has standard deviation pi / (k sqrt 6), so
    k0 = pi / (sqrt 6 * weighted sd of log y)."""
    Nj = w.sum()
    ly = np.log(y)
    mlog = np.sum(w * ly) / Nj
    sdlog = math.sqrt(np.sum(w * (ly - mlog) ** 2) / Nj)
    k = math.pi / (math.sqrt(6.0) * sdlog)
    lmax = ly.max()

    def sums(k):
        e = np.exp(k * (ly - lmax))            # y^k / ymax^k, ratios invariant
        return np.sum(w * e), np.sum(w * e * ly), np.sum(w * e * ly * ly)

    iters = 0
    for iters in range(1, NEWTON_MAXIT + 1):
        S0, S1, S2 = sums(k)
        f = 1.0 / k + mlog - S1 / S0
        df = -1.0 / (k * k) - (S2 * S0 - S1 * S1) / (S0 * S0)
        new = _positive_step(k, f / df)
        done = _newton_done(k, new)
        k = new
        if done:
            break
    S0 = np.sum(w * np.exp(k * ly))
    lam = (S0 / Nj) ** (1.0 / k)
    return dict(k=k, lam=lam, _iters=iters)


def mstep_negbin(w, y, cur):
    """Sec. 4.2 (negative binomial).  The paper gives no score; reading:
    with p = r / (r + ybar) profiled out, Newton on
      g(r)  = sum w [psi(y+r) - psi(r)] + N log(r / (r + ybar)) = 0,
      g'(r) = sum w [psi'(y+r) - psi'(r)] + N (1/r - 1/(r + ybar)),
    seeded at ybar^2 / (var - ybar); when var <= ybar there is no finite
    maximiser and r = 1e6.  Steps are halved to keep r > 0, r <= 1e6."""
    Nj = w.sum()
    ybar = np.sum(w * y) / Nj
    var = np.sum(w * (y - ybar) ** 2) / Nj
    iters = 0
    if var <= ybar:
        r = NEGBIN_RMAX
    else:
        r = ybar * ybar / (var - ybar)
        for iters in range(1, NEWTON_MAXIT + 1):
            g = np.sum(w * (digamma(y + r) - digamma(r))) + Nj * np.log(r / (r + ybar))
            dg = (np.sum(w * (trigamma(y + r) - trigamma(r)))
                  + Nj * (1.0 / r - 1.0 / (r + ybar)))
            new = min(_positive_step(r, g / dg), NEGBIN_RMAX)
            done = _newton_done(r, new)
            r = new
            if done:
                break
    return dict(r=r, p=r / (r + ybar), _iters=iters)


def mstep_vonmises(w, y, cur):
    """Sec. 4.1 mean direction mu = atan2(sum w sin y, sum w cos y);
    Sec. 4.2 Eq. 12: Newton on A(kappa) = Rbar from the seed
    Rbar (2 - Rbar^2) / (1 - Rbar^2)."""
    Nj = w.sum()
    C, S = np.sum(w * np.cos(y)), np.sum(w * np.sin(y))
    mu = math.atan2(S, C)
    R = math.hypot(C, S) / Nj
    if R >= 1.0:
        return dict(mu=mu, kappa=KAPPA_MAX, _iters=0)
    k = R * (2 - R * R) / (1 - R * R)
    iters = 0
    for iters in range(1, NEWTON_MAXIT + 1):
        A = bessel_ratio(k)
        dA = 1 - A * A - A / k
        new = min(_positive_step(k, (A - R) / dA), KAPPA_MAX)
        done = _newton_done(k, new)
        k = new
        if done:
            break
    return dict(mu=mu, kappa=k, _iters=iters)


def student_t_utilde(y, mu, s2, nu):
    """Eq. 14: u_t = (nu + 1) / (nu + (y - mu)^2 / sigma^2)."""
    return (nu + 1) / (nu + (y - mu) ** 2 / s2)


def mstep_student_t(w, y, cur, nu_mode="ecm"):
    """Sec. 4.3.  E-step weights u_t from the current (mu0, sigma0^2, nu0)
    (Eq. 14); CM-step 1 (Eq. 15-16) with sigma^2 divided by N_j and the new
    mu; CM-step 2: Newton on the nu score with the Hessian of Eq. 19 until
    |d nu| < 1e-6.

    nu_mode='ecm' (default reading): the score of Eq. 18 plus the constant
    (N/2)[psi((nu0+1)/2) - log((nu0+1)/2)] that E[log U | y] contributes in
    the ECM equation for nu; Eq. 17-18 as printed omit it, which biases nu
    upward.  nu_mode='paper_literal' uses Eq. 18 exactly as printed.
    nu is kept in [0.5, 1e4] (reading)."""
    mu0, s20, nu0 = cur["mu"], cur["sigma2"], cur["nu"]
    Nj = w.sum()
    u = student_t_utilde(y, mu0, s20, nu0)
    wu = w * u
    mu = np.sum(wu * y) / np.sum(wu)                      # Eq. 15
    s2 = np.sum(wu * (y - mu) ** 2) / Nj                  # Eq. 16
    if s2 <= VAR_RESOLUTION * np.sum(wu * (y - mu0) ** 2) / Nj:
        s2 = 0.0                    # reading 14: undefined, theta_j kept
    C = np.sum(w * (np.log(u) - u))
    if nu_mode == "ecm":
        C += Nj * (digamma((nu0 + 1) / 2) - np.log((nu0 + 1) / 2))
    elif nu_mode != "paper_literal":
        raise ValueError(nu_mode)
    nu = nu0
    iters = 0
    for iters in range(1, NEWTON_MAXIT + 1):
        g = 0.5 * Nj * (np.log(nu / 2) + 1 - digamma(nu / 2)) + 0.5 * C   # Eq. 18
        h = 0.25 * Nj * (2.0 / nu - trigamma(nu / 2))                     # Eq. 19
        dnu = -g / h
        new = min(max(nu + dnu, NU_MIN), NU_MAX)
        done = abs(new - nu) < NU_TOL
        nu = new
        if done:
            break
    return dict(mu=mu, sigma2=s2, nu=nu, _iters=iters)


def mstep_diag_gauss(w, y, cur):
    """Sec. 4.5, Eq. 21: D independent weighted Gaussian updates."""
    Nj = w.sum()
    mu = np.sum(w[:, None] * y, axis=0) / Nj
    var = np.sum(w[:, None] * (y - mu) ** 2, axis=0) / Nj
    return dict(mu=mu, var=var)


def mstep_discrete(w, y, cur):
    """Sec. 4, Discrete (categorical): p_jk = N_j^-1 sum_t gamma_t(j) 1[y_t = k]."""
    K = np.asarray(cur["p"]).shape[0]
    Nj = w.sum()
    counts = np.array([np.sum(w[y == k]) for k in range(K)])
    return dict(p=counts / Nj)


def mstep_full_gauss(w, y, cur):
    """Sec. 4.5, Eq. 23-24: weighted mean and covariance + eps I."""
    Nj = w.sum()
    mu = np.sum(w[:, None] * y, axis=0) / Nj
    d = y - mu
    cov = (w[:, None] * d).T @ d / Nj + TIKHONOV_EPS * np.eye(y.shape[1])
    return dict(mu=mu, cov=cov)


def _safe_log(y):
    """log y where y > 0, else 0 (rows outside the support carry weight 0)."""
    return np.log(np.where(y > 0, y, 1.0))


def mstep_lognormal(w, y, cur):
    """Sec. 4.1 "Log-normal": the Gaussian M-step applied to log y."""
    Nj = w.sum()
    ly = _safe_log(y)
    mu = np.sum(w * ly) / Nj
    s2 = np.sum(w * (ly - mu) ** 2) / Nj
    if s2 <= VAR_RESOLUTION * np.sum(w * (ly - cur.get("mu", mu)) ** 2) / Nj:
        s2 = 0.0                    # reading 14: undefined, theta_j kept
    return dict(mu=mu, sigma2=s2)


def mstep_exponential(w, y, cur):
    """Sec. 4.1 "Exponential": lambda = 1 / ybar_j."""
    return dict(lam=w.sum() / np.sum(w * y))


def mstep_rayleigh(w, y, cur):
    """Sec. 4.1 "Rayleigh": sigma^2 = (2 N_j)^-1 sum_t gamma_t(j) y_t^2."""
    return dict(sigma2=np.sum(w * y * y) / (2 * w.sum()))


def support_rows(family, y, cur):
    """Reading of the min / max in the Uniform and Pareto M-steps (Sec. 4,
    Sec. 4.2): taken over the rows the state can emit under its current
    parameters, {t : b_j(y_t) > 0}.  These are the rows with gamma_t(j) > 0
    whenever pi and A are strictly positive, and the maximiser of Eq. 6 must
    keep every such row inside the new support; the test is exact in any
    precision (a comparison of y with the current bounds)."""
    if family == "uniform":
        return (y >= cur["a"]) & (y <= cur["b"])
    if family == "pareto":
        return y >= cur["xm"]
    raise ValueError(family)


def mstep_uniform(w, y, cur):
    """Sec. 4.1 "Uniform": a = min_t y_t, b = max_t y_t over the state's rows."""
    sel = support_rows("uniform", y, cur)
    if not sel.any():
        return dict(a=np.nan, b=np.nan)
    return dict(a=np.min(y[sel]), b=np.max(y[sel]))


def mstep_chisq(w, y, cur):
    """Sec. 4.2 "Chi-squared": the Gamma M-step with alpha = nu/2 and rate
    beta = 1/2 fixed, optimised over nu alone.  The weighted score in
    x = nu/2 is N_j (mean_w log y - log 2 - digamma(x)); digamma increases
    from -inf to +inf on (0, inf), so the root is unique; it is bracketed
    and found by Brent's method (a library root finder)."""
    from scipy.optimize import brentq
    Nj = w.sum()
    c = np.sum(w * _safe_log(y)) / Nj - np.log(2.0)
    lo, hi = 1e-12, 1.0
    while sp.digamma(hi) < c:
        hi *= 2.0
        if hi > 1e300:
            return dict(nu=np.nan)
    if sp.digamma(lo) > c:
        return dict(nu=np.nan)
    x = brentq(lambda v: sp.digamma(v) - c, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)
    return dict(nu=2.0 * x)


def mstep_pareto(w, y, cur):
    """Sec. 4.2 "Pareto": xm = min_t y_t over the state's rows (the
    constrained MLE), then alpha = N_j / sum_t gamma_t(j) log(y_t / xm)."""
    sel = support_rows("pareto", y, cur)
    if not sel.any():
        return dict(xm=np.nan, alpha=np.nan)
    xm = np.min(y[sel])
    Nj = w.sum()
    return dict(xm=xm, alpha=Nj / (np.sum(w * _safe_log(y)) - Nj * np.log(xm)))


MSTEP = dict(gauss=mstep_gauss, poisson=mstep_poisson, gamma=mstep_gamma,
             beta=mstep_beta, weibull=mstep_weibull, negbin=mstep_negbin,
             student_t=mstep_student_t, vonmises=mstep_vonmises,
             diag_gauss=mstep_diag_gauss, full_gauss=mstep_full_gauss, discrete=mstep_discrete,
             lognormal=mstep_lognormal, exponential=mstep_exponential, rayleigh=mstep_rayleigh,
             uniform=mstep_uniform, chisq=mstep_chisq, pareto=mstep_pareto)


def _state_params(model: Model, j: int) -> dict:
    return {k: v[j] for k, v in model.params.items()}


def mstep_emission(model: Model, W: np.ndarray, y: np.ndarray, nu_mode="ecm"):
    """Eq. 6 for every state with the Sec. 4.4 collapse guard.
    W: [T_total, N] occupancies, y: observations of the same rows."""
    new = model.copy()
    iters = np.zeros(model.n_states, dtype=np.int64)
    if model.family == "indep":
        # Sec. 4.5: each component's scalar M-step with the same weights;
        # rows of zero weight (outside some component's support) add nothing
        y = np.asarray(y, dtype=np.float64).reshape(len(W), -1)
        for j in range(model.n_states):
            w = W[:, j]
            if w.sum() < COLLAPSE_EPS:          # Sec. 4.4: keep theta_j
                continue
            rows = w > 0
            for d, fam in enumerate(model.components):
                cm = component_model(model, d)
                kw = dict(nu_mode=nu_mode) if fam == "student_t" else {}
                with np.errstate(all="ignore"):
                    res = MSTEP[fam](w[rows], y[rows, d], _state_params(cm, j), **kw)
                iters[j] += res.pop("_iters", 0)
                if not valid_update(fam, res):   # undefined update keeps the component
                    continue
                for k, v in res.items():
                    new.params[f"d{d}.{k}"][j] = v
        return new, iters
    for j in range(model.n_states):
        w = W[:, j]
        if w.sum() < COLLAPSE_EPS:              # Sec. 4.4: keep theta_j
            continue
        fn = MSTEP[model.family]
        kw = dict(nu_mode=nu_mode) if model.family == "student_t" else {}
        with np.errstate(all="ignore"):
            res = fn(w, y, _state_params(model, j), **kw)
        iters[j] = res.pop("_iters", 0)
        if not valid_update(model.family, res):   # reading: undefined update keeps theta_j
            continue
        for k, v in res.items():
            new.params[k][j] = v
    return new, iters


def valid_update(family, res) -> bool:
    """Reading (extends the Sec. 4.4 collapse guard): an M-step result that is
    not finite or leaves the family's parameter domain (a zero weighted
    variance, a covariance that is not positive definite) is undefined on
    the state's data, and the state keeps its parameters."""
    vals = {k: np.asarray(v, dtype=np.float64) for k, v in res.items()}
    if not all(np.all(np.isfinite(v)) for v in vals.values()):
        return False
    positive = {"gauss": ("sigma2",), "poisson": ("lam",), "gamma": ("alpha", "beta"),
                "beta": ("a", "b"), "weibull": ("k", "lam"), "negbin": ("r",),
                "student_t": ("sigma2", "nu"), "vonmises": (), "diag_gauss": ("var",),
                "lognormal": ("sigma2",), "exponential": ("lam",), "rayleigh": ("sigma2",),
                "chisq": ("nu",), "pareto": ("xm", "alpha")}
    for k in positive.get(family, ()):
        if not np.all(vals[k] > 0):
            return False
    if family == "vonmises" and not np.all(vals["kappa"] >= 0):
        return False
    if family == "negbin" and not (0 < vals["p"] < 1):
        return False
    if family == "discrete" and not (np.all(vals["p"] >= 0) and abs(vals["p"].sum() - 1) < 1e-9):
        return False
    if family == "uniform" and not vals["a"] < vals["b"]:
        return False
    if family == "full_gauss":
        try:
            np.linalg.cholesky(vals["cov"])
        except np.linalg.LinAlgError:
            return False
    return True


def mstep_transitions(model: Model, xi_sum, gamma1_sum, n_seq, alpha_A=1.0, alpha_pi=1.0):
    """Reading (the paper names Baum-Welch but prints no transition update):
    a_ij = sum xi(i,j) / sum_j' xi(i,j') (the denominator equals
    sum_{t<T} gamma_t(i)); a row whose denominator is below 1e-8 is kept
    (the Sec. 4.4 rule applied to rows); pi_j = mean over the model's
    sequences of gamma_1(j).

    MAP Baum-Welch (the paper names a MAP trainer, Sec. 5.6, without a
    definition; reading): symmetric Dirichlet priors Dir(alpha_A) on every
    row of A and Dir(alpha_pi) on pi, flat priors on the emission
    parameters; the M-step takes the posterior mode, i.e. adds the
    pseudo-counts alpha - 1 (alpha <= 1 adds none):
    a_ij = (n_ij + alpha_A - 1) / (sum_j' n_ij' + N (alpha_A - 1)),
    pi_j = (sum_s gamma_1(j) + alpha_pi - 1) / (S + N (alpha_pi - 1))."""
    N = model.n_states
    cA = max(alpha_A - 1.0, 0.0)
    cp = max(alpha_pi - 1.0, 0.0)
    A = model.A.copy()
    num = xi_sum + cA
    den = num.sum(axis=1)
    for i in range(N):
        if den[i] >= COLLAPSE_EPS:
            A[i] = num[i] / den[i]
    pi = (gamma1_sum + cp) / (n_seq + N * cp)
    return pi, A


def log_dirichlet_prior(model: Model, alpha_A=1.0, alpha_pi=1.0) -> float:
    """log of the (unnormalised) Dirichlet prior density of the MAP reading
    at the model's pi and A: sum (alpha - 1) log p."""
    cA = max(alpha_A - 1.0, 0.0)
    cp = max(alpha_pi - 1.0, 0.0)
    with np.errstate(divide="ignore"):
        return float(cA * np.sum(np.log(model.A)) + cp * np.sum(np.log(model.pi)))


# --------------------------------------------------------------------------
# One Baum-Welch iteration over a packed ragged batch of several models
# --------------------------------------------------------------------------
def split_batch(values, offsets):
    return [values[offsets[s]:offsets[s + 1]] for s in range(len(offsets) - 1)]


def estep(models, values, offsets, model_id):
    """Per model: per-sequence logL, occupancies of every row of its data,
    sum of xi, sum of gamma_1 and the number of sequences."""
    seqs = split_batch(values, offsets)
    out = []
    for m, model in enumerate(models):
        idx = [s for s in range(len(seqs)) if model_id[s] == m]
        N = model.n_states
        res = dict(seq=idx, logL=[], W=[], Y=[], xi_sum=np.zeros((N, N)),
                   gamma1_sum=np.zeros(N), n_seq=len(idx))
        for s in idx:
            fb = forward_backward(model, seqs[s])
            res["logL"].append(fb["logL"])
            res["W"].append(fb["gamma"])
            res["Y"].append(seqs[s])
            res["xi_sum"] += fb["xi_sum"]
            res["gamma1_sum"] += fb["gamma"][0]
        out.append(res)
    return out


def em_iteration(models, values, offsets, model_id, nu_mode="ecm", alpha_A=1.0, alpha_pi=1.0):
    """E-step with the current models, then the M-step of Sec. 4 for the
    emissions and the transition/initial reading (with alpha_A / alpha_pi
    > 1: the MAP reading of mstep_transitions).  Returns
    (new_models, logL per sequence [S] under the OLD models)."""
    S = len(offsets) - 1
    logL = np.zeros(S)
    new_models = []
    for model, res in zip(models, estep(models, values, offsets, model_id)):
        for s, ll in zip(res["seq"], res["logL"]):
            logL[s] = ll
        if res["n_seq"] == 0:
            new_models.append(model.copy())
            continue
        W = np.concatenate(res["W"], axis=0)
        Y = np.concatenate(res["Y"], axis=0)
        new, _ = mstep_emission(model, W, Y, nu_mode=nu_mode)
        new.pi, new.A = mstep_transitions(model, res["xi_sum"],
                                          res["gamma1_sum"], res["n_seq"], alpha_A, alpha_pi)
        new_models.append(new)
    return new_models, logL


# --------------------------------------------------------------------------
# Viterbi training (the paper names a Viterbi trainer, Sec. 5.6, without a
# definition; reading: segmental k-means / hard EM).  The E-step decodes
# each sequence's Viterbi path q* (Eq. 3-4) and replaces the posteriors by
# the path's indicators, gamma_t(j) = 1[q*_t = j] and
# xi_t(i,j) = 1[q*_t = i, q*_{t+1} = j]; the M-step is the Baum-Welch one on
# these weights.  The objective sum_s max_q log P(q, y_s) does not decrease:
# the M-step maximises log P(q*, y) over the parameters for the fixed paths,
# and decoding again can only raise the maximum over q.
# --------------------------------------------------------------------------
def viterbi_estep(models, values, offsets, model_id):
    """Per model: the hard occupancies of every row of its data, transition
    counts, first-state counts, the number of sequences, and per sequence
    the Viterbi path and its score."""
    seqs = split_batch(values, offsets)
    out = []
    for m, model in enumerate(models):
        idx = [s for s in range(len(seqs)) if model_id[s] == m]
        N = model.n_states
        res = dict(seq=idx, score=[], path=[], W=[], Y=[], xi_sum=np.zeros((N, N)),
                   gamma1_sum=np.zeros(N), n_seq=len(idx))
        for s in idx:
            y = seqs[s]
            if len(y) == 0:
                res["score"].append(0.0)
                res["path"].append(np.zeros(0, np.int32))
                continue
            q, sc = viterbi(model, y)
            W = np.zeros((len(y), N))
            W[np.arange(len(y)), q] = 1.0
            np.add.at(res["xi_sum"], (q[:-1], q[1:]), 1.0)
            res["gamma1_sum"][q[0]] += 1.0
            res["score"].append(sc)
            res["path"].append(q)
            res["W"].append(W)
            res["Y"].append(y)
        out.append(res)
    return out


def viterbi_train_iteration(models, values, offsets, model_id, nu_mode="ecm"):
    """One Viterbi-training iteration; returns (new_models, the Viterbi
    score of every sequence [S] under the OLD models)."""
    S = len(offsets) - 1
    score = np.zeros(S)
    new_models = []
    for model, res in zip(models, viterbi_estep(models, values, offsets, model_id)):
        for s, sc in zip(res["seq"], res["score"]):
            score[s] = sc
        if not res["W"]:
            new_models.append(model.copy())
            continue
        new, _ = mstep_emission(model, np.concatenate(res["W"]), np.concatenate(res["Y"]), nu_mode=nu_mode)
        new.pi, new.A = mstep_transitions(model, res["xi_sum"], res["gamma1_sum"], res["n_seq"])
        new_models.append(new)
    return new_models, score


def fit(models, values, offsets, model_id, n_iter, nu_mode="ecm"):
    """n_iter Baum-Welch iterations; returns (models, logL trace
    [n_iter, S]) where row k holds the logL under the models entering
    iteration k."""
    trace = []
    for _ in range(n_iter):
        models, ll = em_iteration(models, values, offsets, model_id, nu_mode)
        trace.append(ll)
    return models, np.array(trace)


def free_parameter_count(model: Model) -> int:
    """Free parameters of an HMM, counted from its parameter arrays: the
    N - 1 free initial probabilities, N (N - 1) free transition
    probabilities, and every emission parameter entry except those fixed by
    a constraint (a probability row sums to 1; a covariance matrix is
    symmetric)."""
    N = model.n_states
    k = (N - 1) + N * (N - 1)
    for name, v in model.params.items():
        v = np.asarray(v)
        if model.family == "discrete" and name == "p":          # rows on the simplex
            k += v.shape[0] * (v.shape[1] - 1)
        elif model.family == "full_gauss" and name == "cov":    # symmetric D x D
            D = v.shape[1]
            k += v.shape[0] * D * (D + 1) // 2
        else:
            k += v.size
    return k


def information_criteria(model: Model, logL: float, n_obs: int) -> dict:
    """AIC, BIC and AICc (named by the paper for model comparison, no formula
    printed): the textbook definitions 2k - 2 logL, k ln n - 2 logL and
    AIC + 2k(k+1)/(n-k-1) (infinite when n <= k + 1)."""
    k = free_parameter_count(model)
    aic = 2 * k - 2 * logL
    bic = k * math.log(n_obs) - 2 * logL
    aicc = aic + 2 * k * (k + 1) / (n_obs - k - 1) if n_obs - k - 1 > 0 else math.inf
    return dict(k=k, aic=aic, bic=bic, aicc=aicc)


def batch_loglik(models, values, offsets, model_id):
    seqs = split_batch(values, offsets)
    return np.array([forward_backward(models[model_id[s]], seqs[s])["logL"]
                     for s in range(len(seqs))])


# --------------------------------------------------------------------------
# Brute force over all N^T state paths (tiny N, T) -- pins the recursions
# --------------------------------------------------------------------------
def brute_force(logpi, logA, logb):
    """Enumerate every path q in [N]^T: returns logL, gamma, sum xi, the
    MAP path (lowest path in lexicographic order among exact ties) and its
    score.  Exponential cost; N <= 3, T <= 8 only."""
    import itertools
    T, N = logb.shape
    paths = np.array(list(itertools.product(range(N), repeat=T)))
    lp = logpi[paths[:, 0]] + logb[0, paths[:, 0]]
    for t in range(1, T):
        lp = lp + logA[paths[:, t - 1], paths[:, t]] + logb[t, paths[:, t]]
    logL = float(lse(lp, axis=0))
    post = np.exp(lp - logL)
    gamma = np.zeros((T, N))
    xi = np.zeros((N, N))
    for t in range(T):
        np.add.at(gamma[t], paths[:, t], post)
    for t in range(T - 1):
        np.add.at(xi, (paths[:, t], paths[:, t + 1]), post)
    best = int(np.argmax(lp))
    return dict(logL=logL, gamma=gamma, xi_sum=xi,
                map_path=paths[best].astype(np.int32), map_score=float(lp[best]),
                all_scores=lp, paths=paths)


# --------------------------------------------------------------------------
# k-means++ seeding and Lloyd iterations (Sec. 4.5 initialisation; the paper
# gives no constants).  Reading: features are float32 values computed in
# float64; the uniforms u_0..u_{K-1} in [0, 1) are inputs.  The first
# centre is the observation floor(u_0 T); centre j is the first observation
# i whose running sum of D2 (the squared distance to the nearest centre so
# far) exceeds u_j times the total (if the total is 0: floor(u_j T)).  Lloyd
# iterations assign every observation to its nearest centre (the lowest
# index at ties) and move every non-empty cluster's centre to the mean of
# its observations, until no assignment changes or max_iter assignment
# passes.
# --------------------------------------------------------------------------
def kmeanspp(X, u, max_iter=100):
    """Returns (centres [K, F] float64, labels [T] int32, assignment passes)."""
    X = np.asarray(X, dtype=np.float64)
    X = X[:, None] if X.ndim == 1 else X
    T, F = X.shape
    K = len(u)
    C = np.empty((K, F))
    C[0] = X[min(int(math.floor(u[0] * T)), T - 1)]
    d2 = np.sum((X - C[0]) ** 2, axis=1)
    for j in range(1, K):
        tot = float(np.sum(d2))
        if tot > 0:
            cum = np.cumsum(d2)
            i = int(np.searchsorted(cum, u[j] * tot, side="right"))
            i = min(i, T - 1)
        else:
            i = min(int(math.floor(u[j] * T)), T - 1)
        C[j] = X[i]
        d2 = np.minimum(d2, np.sum((X - C[j]) ** 2, axis=1))
    labels = None
    passes = 0
    for passes in range(1, max_iter + 1):
        dist = np.sum((X[:, None, :] - C[None, :, :]) ** 2, axis=2)
        new = np.argmin(dist, axis=1).astype(np.int32)     # first minimum: lowest index
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for j in range(K):
            sel = labels == j
            if sel.any():
                C[j] = X[sel].mean(axis=0)
    return C, labels, passes
