import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def as_oracle_model(d):
    from oracle import hmm_oracle as O
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(),
                   {k: v.copy() for k, v in d["params"].items()})


def pytest_terminal_summary(terminalreporter):
    """Logs every Viterbi near-tie site the GPU parity tests excused (a
    device path that differs from the float64 oracle's within the score-gap
    bar)."""
    try:
        import parity
    except ImportError:
        return
    if parity.NEAR_TIES:
        terminalreporter.write_line(f"viterbi near-ties excused: {len(parity.NEAR_TIES)}")
        for where, n_diff, gap in parity.NEAR_TIES:
            terminalreporter.write_line(f"  {where}: {n_diff} steps differ, float64 score gap {gap:.3e}")
