"""ctypes declarations of the hmmgpu C ABI (include/hmmgpu.h)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

HMM_OK = 0
STATUS_NAMES = {0: "HMM_OK", 1: "HMM_E_ARG", 2: "HMM_E_NOMEM", 3: "HMM_E_CUDA",
                4: "HMM_E_NUMERIC", 5: "HMM_E_TIMEOUT", 6: "HMM_E_BUSY",
                7: "HMM_E_NOTREADY", 8: "HMM_E_UNSUPPORTED"}

OPT_PROFILE, OPT_ESTEP_LANES, OPT_VITERBI_LANES, OPT_PLAIN_ESTEP, OPT_TENSOR_RECURRENCE = 1, 2, 3, 4, 5
OPT_TIME_PARALLEL = 6
# values of OPT_TENSOR_RECURRENCE: float32 CUDA cores, FP16 tensor cores, TF32 (padded N <= 256)
TENSOR_REC_OFF, TENSOR_REC_FP16, TENSOR_REC_TF32 = 0, 1, 2
KT_SLOTS = ("estep", "reduce", "mstep", "viterbi", "emission", "plain", "xi", "slot7")

FAMILY = {"gauss": 0, "poisson": 1, "gamma": 2, "beta": 3, "weibull": 4, "negbin": 5,
          "student_t": 6, "vonmises": 7, "diag_gauss": 8, "full_gauss": 9, "discrete": 10,
          "lognormal": 11, "exponential": 12, "rayleigh": 13, "uniform": 14, "chisq": 15, "pareto": 16,
          "indep": 17}


class hmm_batch(C.Structure):
    _fields_ = [("values", C.c_void_p), ("offsets", C.c_void_p), ("model_id", C.c_void_p),
                ("n_seq", C.c_int64), ("total_T", C.c_int64), ("dim", C.c_int32),
                ("plan", C.c_void_p)]


class hmm_mstep_opts(C.Structure):
    _fields_ = [("collapse_eps", C.c_double), ("tikhonov_eps", C.c_double),
                ("newton_maxit", C.c_int32), ("newton_tol", C.c_double),
                ("nu_mode", C.c_int32), ("update_transitions", C.c_int32),
                ("dirichlet_A", C.c_double), ("dirichlet_pi", C.c_double)]


class hmm_fit_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("tol", C.c_double), ("mstep", hmm_mstep_opts),
                ("trainer", C.c_int32)]


class hmm_serve_opts(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("max_batch", C.c_int32), ("max_queue", C.c_int32),
                ("mem_budget", C.c_size_t)]


class hmm_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("family", C.c_int32), ("n_states", C.c_int32), ("dim", C.c_int32),
                ("params", C.c_void_p), ("n_params", C.c_int64), ("values", C.c_void_p), ("T", C.c_int64),
                ("n_iter", C.c_int32)]


class hmm_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("T", C.c_int64), ("loglik", C.c_double),
                ("score", C.c_double), ("path", C.POINTER(C.c_int32)), ("gamma", C.POINTER(C.c_float)),
                ("params", C.POINTER(C.c_double)), ("trace", C.POINTER(C.c_double)), ("n_iter", C.c_int32),
                ("latency_ms", C.c_double), ("error", C.c_char_p)]


REQ_DECODE, REQ_POSTERIOR, REQ_FIT = 0, 1, 2
REDUCE_SUM_F64, REDUCE_MIN_I32 = 0, 1
# hmm_allreduce_fn: (d_values, n, op, stream, user) -> 0 on success
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p)

# name -> (restype, argtypes)
_SIGS = {
    "hmm_status_string": (C.c_char_p, [C.c_int]),
    "hmm_last_error": (C.c_char_p, []),
    "hmm_version": (C.c_char_p, []),
    "hmm_family_param_count": (C.c_int32, [C.c_int32, C.c_int32]),
    "hmm_param_blob_size": (C.c_int64, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "hmm_information_criteria": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int64, C.c_void_p]),
    "hmm_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]),
    "hmm_ctx_destroy": (C.c_int, [C.c_void_p]),
    "hmm_ctx_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "hmm_ctx_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "hmm_ctx_wait_selftest": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
    "hmm_ctx_profile_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "hmm_model_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "hmm_model_create_indep": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                         C.POINTER(C.c_void_p)]),
    "hmm_model_blob_size": (C.c_int64, [C.c_void_p]),
    "hmm_model_destroy": (C.c_int, [C.c_void_p]),
    "hmm_model_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "hmm_model_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "hmm_kmeans": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                             C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hmm_plan_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p,
                                  C.c_void_p, C.POINTER(C.c_void_p)]),
    "hmm_plan_destroy": (C.c_int, [C.c_void_p]),
    "hmm_plan_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p, C.c_void_p]),
    "hmm_emission_logpdf": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p,
                                      C.c_void_p]),
    "hmm_forward_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hmm_forward_backward_static": (C.c_int, [C.c_void_p, C.POINTER(hmm_batch), C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p]),
    "hmm_viterbi": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "hmm_stats_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "hmm_stats_destroy": (C.c_int, [C.c_void_p]),
    "hmm_stats_size": (C.c_int64, [C.c_void_p]),
    "hmm_stats_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "hmm_stats_device_buffer": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "hmm_stats_set_allreduce": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hmm_stats_record": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32)]),
    "hmm_estep_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "hmm_estep_viterbi": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "hmm_mstep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(hmm_batch),
                            C.POINTER(hmm_mstep_opts), C.c_void_p]),
    "hmm_fit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(hmm_batch), C.POINTER(hmm_fit_opts),
                          C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    "hmm_serve_create": (C.c_int, [C.c_void_p, C.POINTER(hmm_serve_opts), C.POINTER(C.c_void_p)]),
    "hmm_serve_submit": (C.c_int, [C.c_void_p, C.POINTER(hmm_request), C.POINTER(C.c_uint64)]),
    "hmm_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(hmm_result)]),
    "hmm_serve_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(hmm_result)]),
    "hmm_serve_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "hmm_serve_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "hmm_serve_destroy": (C.c_int, [C.c_void_p]),
}

# every symbol the header declares (checked by the not-gpu tests)
EXPORTED = tuple(_SIGS)

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libhmmgpu.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"hmmgpu library not built ({path}); run paper_2605_29208_gb300.build.build()")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int):
    if status != HMM_OK:
        raise HmmError(status, _lib.hmm_last_error().decode())
