"""hmmgpu: the data-parallel HMM hot path (Baum-Welch and Viterbi) on a
GB300 GPU (sm_103a), behind a C ABI (include/hmmgpu.h).

This module is argument marshalling only: every step of the computation
runs in the CUDA kernels of ``libhmmgpu.so``.  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing the wrappers on a
machine without the built library, or calling them without a GPU, raises.

Typical use (models are dicts: family, pi [N], A [N, N], params {name:
array}; a batch is the packed ragged layout: values, offsets [S + 1],
model_id [S])::

    import paper_2605_29208_gb300 as H
    ctx = H.Context(0)
    model = H.Model(ctx, [start_model])             # one or many models
    batch = H.Batch(values, offsets, model_id).make_plan(ctx, model)
    trace, n_done = H.fit(ctx, model, batch, n_iter=20)    # Baum-Welch
    loglik, gamma, _ = H.forward_backward(ctx, model, batch)
    path, score = H.viterbi(ctx, model, batch)
    fitted = model.get()

Starting models: ``initialize.kmeanspp_init``; restarts and state-count
selection in one batch: ``restarts.fit_restarts`` / ``restarts.select_states``;
a request server with continuous batching: ``Server``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import FAMILY, HmmError, check

__all__ = ["Context", "Model", "Batch", "FAMILY", "HmmError", "blob_from_model",
           "model_from_blob", "information_criteria"]


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


PARAM_ORDER = {
    "gauss": ("mu", "sigma2"), "poisson": ("lam",), "gamma": ("alpha", "beta"),
    "beta": ("a", "b"), "weibull": ("k", "lam"), "negbin": ("r", "p"),
    "student_t": ("mu", "sigma2", "nu"), "vonmises": ("mu", "kappa"),
    "diag_gauss": ("mu", "var"), "full_gauss": ("mu", "cov"), "discrete": ("p",),
    "lognormal": ("mu", "sigma2"), "exponential": ("lam",), "rayleigh": ("sigma2",),
    "uniform": ("a", "b"), "chisq": ("nu",), "pareto": ("xm", "alpha"),
}


def _state_names(model: dict) -> list[str]:
    """Parameter names of one state in blob order (independent components:
    "d<k>.<name>" for every component k in order)."""
    if model["family"] == "indep":
        return [f"d{d}.{n}" for d, f in enumerate(model["components"]) for n in PARAM_ORDER[f]]
    return list(PARAM_ORDER[model["family"]])


def blob_from_model(model: dict) -> np.ndarray:
    """Flattens a model dict {family, pi, A, params} into the C-ABI blob
    (pi, A, then per state its family parameters)."""
    N = len(model["pi"])
    parts = [np.asarray(model["pi"], np.float64).ravel(), np.asarray(model["A"], np.float64).ravel()]
    per_state = []
    for j in range(N):
        for name in _state_names(model):
            per_state.append(np.asarray(model["params"][name][j], np.float64).ravel())
    parts.extend(per_state)
    return np.concatenate(parts)


def model_from_blob(blob: np.ndarray, family: str, N: int, D: int = 1, components=None) -> tuple[dict, int]:
    """Inverse of blob_from_model; returns (model, values consumed)."""
    q = 0
    pi = blob[q:q + N].copy(); q += N
    A = blob[q:q + N * N].reshape(N, N).copy(); q += N * N
    if family == "indep":
        names = _state_names(dict(family="indep", components=components))
        vals = blob[q:q + N * len(names)].reshape(N, len(names)); q += N * len(names)
        return dict(family="indep", components=list(components), pi=pi, A=A,
                    params={n: vals[:, i].copy() for i, n in enumerate(names)}), q
    names = PARAM_ORDER[family]
    sizes = {"mu": D if family in ("diag_gauss", "full_gauss") else 1,
             "var": D, "cov": D * D, "p": D}
    params = {n: [] for n in names}
    for j in range(N):
        for n in names:
            k = sizes.get(n, 1) if family in ("diag_gauss", "full_gauss", "discrete") else 1
            v = blob[q:q + k]; q += k
            params[n].append(v.reshape(D, D) if n == "cov" else (v if k > 1 else v[0]))
    params = {n: np.array(v) for n, v in params.items()}
    return dict(family=family, pi=pi, A=A, params=params), q


class Context:
    """A CUDA device context of the library (owns its scratch memory)."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self.lib = _lib.load()
        h = C.c_void_p()
        check(self.lib.hmm_ctx_create(device, workspace_bytes, C.byref(h)))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.hmm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        return self.lib.hmm_ctx_status(self.h, _stream(stream))

    def set_option(self, key: int, value: int):
        check(self.lib.hmm_ctx_set_option(self.h, key, value))

    def profile(self, reset: bool = False) -> dict:
        """{slot: (milliseconds, launches)} of the kernels timed so far."""
        ms = np.zeros(8, np.float64)
        n = np.zeros(8, np.int64)
        check(self.lib.hmm_ctx_profile_read(self.h, ms.ctypes.data_as(C.c_void_p),
                                            n.ctypes.data_as(C.c_void_p), 8, int(reset)))
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(_lib.KT_SLOTS)}


class Model:
    """M models x N states on the device; ``models`` is a list of model dicts
    that share N (and D)."""

    def __init__(self, ctx: Context, models: list[dict]):
        self.ctx, self.lib = ctx, ctx.lib
        self.families = [m["family"] for m in models]
        self.components = [list(m.get("components", ())) for m in models]
        self.N = len(models[0]["pi"])
        mu = models[0]["params"].get("mu")
        if self.families[0] == "discrete":        # dim = number of symbols
            self.D = int(np.asarray(models[0]["params"]["p"]).shape[1])
        elif self.families[0] == "indep":         # dim = number of components
            self.D = len(self.components[0])
        else:
            self.D = (np.asarray(mu).shape[1] if self.families[0] in ("diag_gauss", "full_gauss") else 1)
        fam = np.array([FAMILY[f] for f in self.families], np.int32)
        h = C.c_void_p()
        if self.families[0] == "indep":
            comp = np.array([[FAMILY[f] for f in c] for c in self.components], np.int32)
            check(self.lib.hmm_model_create_indep(ctx.h, len(models), self.N, self.D,
                                                  comp.ctypes.data_as(C.c_void_p), C.byref(h)))
        else:
            check(self.lib.hmm_model_create(ctx.h, len(models), self.N, self.D,
                                            fam.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.h = h
        self._fam = fam
        self.set(models)

    @property
    def n_models(self):
        return len(self.families)

    def blob_size(self):
        return self.lib.hmm_model_blob_size(self.h)

    def set(self, models: list[dict]):
        blob = np.concatenate([blob_from_model(m) for m in models])
        check(self.lib.hmm_model_set_params(self.h, blob.ctypes.data_as(C.c_void_p), blob.size))

    def get(self) -> list[dict]:
        n = self.blob_size()
        blob = np.empty(n, np.float64)
        check(self.lib.hmm_model_get_params(self.h, blob.ctypes.data_as(C.c_void_p), n))
        out, q = [], 0
        for f, comp in zip(self.families, self.components):
            m, used = model_from_blob(blob[q:], f, self.N, self.D, comp)
            out.append(m)
            q += used
        return out

    def close(self):
        if self.h:
            self.lib.hmm_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A packed ragged batch resident on the device (float32 values, int64
    offsets, int32 model ids) with an optional plan."""

    def __init__(self, values, offsets, model_id, device="cuda", dim=1):
        torch = _torch()
        self.values = torch.as_tensor(np.asarray(values, np.float32)).to(device).contiguous()
        self.offsets = torch.as_tensor(np.asarray(offsets, np.int64)).to(device).contiguous()
        self.model_id = torch.as_tensor(np.asarray(model_id, np.int32)).to(device).contiguous()
        self.h_offsets = np.ascontiguousarray(offsets, np.int64)
        self.h_model_id = np.ascontiguousarray(model_id, np.int32)
        self.n_seq = len(self.h_offsets) - 1
        self.total_T = int(self.h_offsets[-1]) if self.n_seq >= 0 else 0
        self.dim = dim
        self.plan = None
        self._lib = None

    def c(self):
        return _lib.hmm_batch(self.values.data_ptr() if self.values.numel() else None,
                              self.offsets.data_ptr(), self.model_id.data_ptr() if self.n_seq else None,
                              self.n_seq, self.total_T, self.dim, self.plan)

    def make_plan(self, ctx: Context, model: Model):
        b = self.c()
        h = C.c_void_p()
        check(ctx.lib.hmm_plan_create(ctx.h, model.h, C.byref(b),
                                      self.h_offsets.ctypes.data_as(C.c_void_p),
                                      self.h_model_id.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.plan = h
        self._lib = ctx.lib
        return self

    def autotune(self, ctx: Context, model: Model, stream=None):
        """hmm_plan_autotune: pick the fastest chain widths for this batch;
        returns the measured (E-step ms, Viterbi ms)."""
        ms = np.zeros(2, np.float64)
        b = self.c()
        check(ctx.lib.hmm_plan_autotune(ctx.h, model.h, C.byref(b), ms.ctypes.data_as(C.c_void_p),
                                        _stream(stream)))
        return tuple(ms)

    def __del__(self):
        try:
            if self.plan and self._lib:
                self._lib.hmm_plan_destroy(self.plan)
        except Exception:
            pass


# ------------------------------------------------------------------ calls
def information_criteria(family: str, n_states: int, loglik: float, n_obs: int, dim: int = 1) -> dict:
    """hmm_information_criteria: free-parameter count k, AIC, BIC and AICc of
    one fitted model (host arithmetic in the library, no device work)."""
    from . import _lib
    lib = _lib.load()
    out = np.zeros(4, np.float64)
    check(lib.hmm_information_criteria(FAMILY[family], int(n_states), int(dim), float(loglik), int(n_obs),
                                       out.ctypes.data_as(C.c_void_p)))
    return dict(k=int(out[0]), aic=float(out[1]), bic=float(out[2]), aicc=float(out[3]))


def emission_logpdf(ctx, model, batch, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty((batch.total_T, model.N), dtype=torch.float32, device=batch.values.device)
    b = batch.c()
    check(ctx.lib.hmm_emission_logpdf(ctx.h, model.h, C.byref(b), _ptr(out), _stream(stream)))
    return out


def forward_backward(ctx, model, batch, logb=None, want_gamma=True, want_path=False, stream=None):
    torch = _torch()
    dev = batch.values.device
    ll = torch.empty(batch.n_seq, dtype=torch.float64, device=dev)
    gamma = torch.empty((batch.total_T, model.N), dtype=torch.float32, device=dev) if want_gamma else None
    path = torch.empty(batch.total_T, dtype=torch.int32, device=dev) if want_path else None
    b = batch.c()
    check(ctx.lib.hmm_forward_backward(ctx.h, model.h, C.byref(b), _ptr(logb), _ptr(gamma), _ptr(path),
                                       _ptr(ll), _stream(stream)))
    return ll, gamma, path


def forward_backward_static(model, batch, gamma, loglik, logb=None, stream=None):
    """hmm_forward_backward_static: same outputs as forward_backward, written
    into the caller's tensors; the library allocates nothing during the call
    (its scratch is a fixed device array, see include/hmmgpu.h)."""
    b = batch.c()
    check(model.lib.hmm_forward_backward_static(model.h, C.byref(b), _ptr(logb), _ptr(gamma), _ptr(loglik),
                                                _stream(stream)))
    return loglik, gamma


def kmeans(ctx, X, u, max_iter=100, stream=None):
    """hmm_kmeans: k-means++ seeding from the uniforms u [R][K] and Lloyd
    iterations on the device for R restarts of the features X [T][F]
    (float32, a torch tensor on the GPU or an array); returns (centres
    [R][K][F] float64, labels [R][T] int32, passes [R])."""
    torch = _torch()
    X = torch.as_tensor(np.asarray(X, np.float32) if not torch.is_tensor(X) else X).to("cuda", torch.float32)
    X = X.reshape(X.shape[0], -1).contiguous()
    u = np.ascontiguousarray(np.atleast_2d(u), np.float64)
    R, K = u.shape
    T, F = X.shape
    centres = torch.empty((R, K, F), dtype=torch.float64, device=X.device)
    labels = torch.full((R, T), -1, dtype=torch.int32, device=X.device)
    passes = np.zeros(R, np.int32)
    check(ctx.lib.hmm_kmeans(ctx.h, _ptr(X), T, F, K, R, u.ctypes.data_as(C.c_void_p), max_iter, _ptr(centres),
                             _ptr(labels), passes.ctypes.data_as(C.c_void_p), _stream(stream)))
    return centres, labels, passes


def viterbi(ctx, model, batch, logb=None, stream=None):
    torch = _torch()
    dev = batch.values.device
    path = torch.empty(batch.total_T, dtype=torch.int32, device=dev)
    score = torch.empty(batch.n_seq, dtype=torch.float64, device=dev)
    b = batch.c()
    check(ctx.lib.hmm_viterbi(ctx.h, model.h, C.byref(b), _ptr(logb), _ptr(path), _ptr(score),
                              _stream(stream)))
    return path, score


class Stats:
    def __init__(self, ctx, model):
        self.lib = ctx.lib
        h = C.c_void_p()
        check(self.lib.hmm_stats_create(ctx.h, model.h, C.byref(h)))
        self.h = h

    def device_tensor(self):
        """The raw float64 statistic record as a torch tensor that aliases
        the library's device memory (for cross-GPU sums)."""
        torch = _torch()
        ptr = C.c_void_p()
        n = C.c_int64()
        check(self.lib.hmm_stats_device_buffer(self.h, C.byref(ptr), C.byref(n)))

        class _View:
            __cuda_array_interface__ = dict(shape=(n.value,), typestr="<f8", data=(ptr.value, False),
                                            version=2)
        return torch.as_tensor(_View(), device="cuda")

    def get(self) -> np.ndarray:
        n = self.lib.hmm_stats_size(self.h)
        out = np.empty(n, np.float64)
        check(self.lib.hmm_stats_get(self.h, out.ctypes.data_as(C.c_void_p), n))
        return out

    def __del__(self):
        try:
            self.lib.hmm_stats_destroy(self.h)
        except Exception:
            pass


def estep_stats(ctx, model, batch, stats=None, stream=None):
    torch = _torch()
    stats = stats or Stats(ctx, model)
    ll = torch.empty(batch.n_seq, dtype=torch.float64, device=batch.values.device)
    b = batch.c()
    check(ctx.lib.hmm_estep_stats(ctx.h, model.h, C.byref(b), stats.h, _ptr(ll), _stream(stream)))
    return stats, ll


def mstep_opts(nu_mode=0, update_transitions=1, **kw):
    o = _lib.hmm_mstep_opts()
    o.collapse_eps = kw.get("collapse_eps", 0.0)
    o.tikhonov_eps = kw.get("tikhonov_eps", 0.0)
    o.newton_maxit = kw.get("newton_maxit", 0)
    o.newton_tol = kw.get("newton_tol", 0.0)
    o.nu_mode = nu_mode
    o.update_transitions = update_transitions
    o.dirichlet_A = kw.get("dirichlet_A", 0.0)
    o.dirichlet_pi = kw.get("dirichlet_pi", 0.0)
    return o


def mstep(ctx, model, stats, batch=None, opts=None, stream=None):
    o = opts or mstep_opts()
    b = batch.c() if batch is not None else None
    check(ctx.lib.hmm_mstep(ctx.h, model.h, stats.h, C.byref(b) if b is not None else None,
                            C.byref(o), _stream(stream)))


def estep_viterbi(ctx, model, batch, stats=None, stream=None):
    """hmm_estep_viterbi: statistics of the Viterbi paths (Viterbi training);
    returns (stats, per-sequence best-path log-probabilities)."""
    torch = _torch()
    stats = stats or Stats(ctx, model)
    sc = torch.empty(batch.n_seq, dtype=torch.float64, device=batch.values.device)
    b = batch.c()
    check(ctx.lib.hmm_estep_viterbi(ctx.h, model.h, C.byref(b), stats.h, _ptr(sc), _stream(stream)))
    return stats, sc


def fit(ctx, model, batch, n_iter, tol=0.0, opts=None, stream=None, trainer="baum_welch"):
    """hmm_fit: n_iter iterations of Baum-Welch (trainer "baum_welch"; MAP
    with dirichlet_* in opts) or Viterbi training (trainer "viterbi")."""
    o = _lib.hmm_fit_opts()
    o.max_iter = n_iter
    o.tol = tol
    o.trainer = {"baum_welch": 0, "viterbi": 1}[trainer]
    o.mstep = opts or mstep_opts()
    trace = np.zeros((max(n_iter, 1), model.n_models), np.float64)
    done = C.c_int32(0)
    b = batch.c()
    check(ctx.lib.hmm_fit(ctx.h, model.h, C.byref(b), C.byref(o), trace.ctypes.data_as(C.c_void_p),
                          C.byref(done), _stream(stream)))
    return trace[:done.value], done.value


class Server:
    """hmm_serve_*: a request server with continuous batching.  Requests
    carry their own model dict and one host sequence; results come back as
    numpy arrays."""

    KINDS = {"decode": _lib.REQ_DECODE, "posterior": _lib.REQ_POSTERIOR, "fit": _lib.REQ_FIT}

    def __init__(self, ctx: Context, n_slots=0, max_batch=0, max_queue=0, mem_budget=0):
        self.lib = ctx.lib
        self.ctx = ctx
        o = _lib.hmm_serve_opts(n_slots, max_batch, max_queue, mem_budget)
        h = C.c_void_p()
        check(self.lib.hmm_serve_create(ctx.h, C.byref(o), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, kind: str, model: dict, values, n_iter: int = 0) -> int:
        fam = FAMILY[model["family"]]
        N = len(model["pi"])
        vals = np.ascontiguousarray(values, np.float32)
        D = vals.shape[1] if vals.ndim == 2 else 1
        blob = blob_from_model(model)
        r = _lib.hmm_request(self.KINDS[kind], fam, N, D, blob.ctypes.data, blob.size, vals.ctypes.data,
                             vals.shape[0], n_iter)
        t = C.c_uint64()
        check(self.lib.hmm_serve_submit(self.h, C.byref(r), C.byref(t)))
        self._keep[t.value] = (kind, N, D, model["family"])
        return t.value

    def _convert(self, ticket, res):
        kind, N, D, family = self._keep[ticket]
        out = dict(status=res.status, latency_ms=res.latency_ms, loglik=res.loglik)
        if res.status != 0:
            out["error"] = (res.error or b"").decode()
            return out
        T = res.T
        if kind == "decode":
            out["path"] = np.ctypeslib.as_array(res.path, shape=(T,)).copy() if T else np.zeros(0, np.int32)
            out["score"] = res.score
        elif kind == "posterior":
            out["gamma"] = (np.ctypeslib.as_array(res.gamma, shape=(T * N,)).reshape(T, N).copy()
                            if T else np.zeros((0, N), np.float32))
        else:
            n = int(self.lib.hmm_param_blob_size(1, N, D, (C.c_int32 * 1)(FAMILY[family])))
            out["params"] = model_from_blob(np.ctypeslib.as_array(res.params, shape=(n,)).copy(), family, N, D)[0]
            out["trace"] = (np.ctypeslib.as_array(res.trace, shape=(res.n_iter,)).copy()
                            if res.n_iter else np.zeros(0))
        return out

    def poll(self, ticket: int):
        res = _lib.hmm_result()
        st = self.lib.hmm_serve_poll(self.h, ticket, C.byref(res))
        if st == 7:      # HMM_E_NOTREADY
            return None
        check(st)
        return self._convert(ticket, res)

    def wait(self, ticket: int, timeout_ms: float = 600000.0, release: bool = True):
        res = _lib.hmm_result()
        check(self.lib.hmm_serve_wait(self.h, ticket, timeout_ms, C.byref(res)))
        out = self._convert(ticket, res)
        if release:
            check(self.lib.hmm_serve_release(self.h, ticket))
            self._keep.pop(ticket, None)
        return out

    def stats(self) -> dict:
        h = np.zeros(10, np.float64)
        check(self.lib.hmm_serve_stats(self.h, h.ctypes.data_as(C.c_void_p)))
        keys = ("submitted", "completed", "p50_ms", "p99_ms", "mean_ms", "completed_per_s", "pending", "running",
                "batches", "slot_occupancy")
        return dict(zip(keys, h.tolist()))

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmm_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

