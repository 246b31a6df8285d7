"""The C-ABI library builds, loads and exports every symbol the header
declares; host-only entry points answer without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "hmmgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_29208_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    from paper_2605_29208_gb300 import _lib
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), f"{s} not exported"
    assert set(syms) == set(_lib.EXPORTED), set(syms) ^ set(_lib.EXPORTED)


def test_host_only_entry_points(lib):
    assert lib.hmm_status_string(0) == b"ok"
    assert b"sm_103a" in lib.hmm_version()
    assert lib.hmm_family_param_count(0, 1) == 2      # Gaussian mu, sigma2
    assert lib.hmm_family_param_count(6, 1) == 3      # Student-t
    assert lib.hmm_family_param_count(8, 4) == 8      # diagonal Gaussian, D = 4
    assert lib.hmm_family_param_count(9, 3) == 12     # full covariance, D = 3
    assert lib.hmm_family_param_count(42, 1) == -1
    fam = np.array([2, 0], np.int32)
    n = lib.hmm_param_blob_size(2, 3, 1, fam.ctypes.data_as(C.c_void_p))
    assert n == 2 * (3 + 9) + 3 * 2 + 3 * 2


def test_no_gpu_gives_an_error_not_a_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.hmm_ctx_create(0, 0, C.byref(h))
    assert st != 0 and not h.value
    assert len(lib.hmm_last_error()) > 0


def test_blob_round_trip():
    from paper_2605_29208_gb300 import blob_from_model, model_from_blob, synth
    rng = np.random.default_rng(0)
    for fam in ("gauss", "gamma", "student_t", "vonmises", "negbin"):
        m = synth.make_model(fam, np.full(3, 1 / 3), synth.dirichlet_rows(rng, 3, 1.0),
                             **synth.random_params(rng, fam, 3))
        b = blob_from_model(m)
        m2, used = model_from_blob(b, fam, 3)
        assert used == len(b)
        for k in m["params"]:
            np.testing.assert_array_equal(m2["params"][k], m["params"][k])
