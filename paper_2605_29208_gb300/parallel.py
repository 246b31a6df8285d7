"""Data-parallel Baum-Welch across processes (one GPU each, torch.distributed).

Sequences are independent in the E-step (paper Sec. 3), and every statistic
the M-step of Sec. 4 reads is a sum over sequences, a minimum / maximum over
rows (uniform and Pareto supports) or, for the Newton steps that re-read the
data (Weibull shape, Eq. 11; negative-binomial r), a sum over rows per
Newton pass.  Each rank holds a contiguous shard of the sequences; the
library calls the exchange installed here on its own device records at the
points where the M-step needs the combined values (hmm_stats_set_allreduce):
after the E-step on the statistic record, the table-family moment record
and the support extremes, and inside the M-step once per Newton data pass.
Every rank then runs the same M-step and keeps the same model.
"""
from __future__ import annotations

import ctypes as C
import traceback

import numpy as np

from . import _lib

SUM_F64 = _lib.REDUCE_SUM_F64
MIN_I32 = _lib.REDUCE_MIN_I32


def shard(n_seq: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of sequences [lo, hi) owned by `rank`."""
    base, extra = divmod(n_seq, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def device_view(ptr: int, n: int, op: int, device: str = "cuda"):
    """A torch tensor aliasing n elements of library memory at `ptr`, of
    the element type the reduction `op` works on (device memory; host
    memory when device == "cpu")."""
    import torch
    if device == "cpu":
        ctype = C.c_double if op == SUM_F64 else C.c_int32
        buf = (ctype * int(n)).from_address(int(ptr))
        return torch.from_numpy(np.ctypeslib.as_array(buf))
    typestr = "<f8" if op == SUM_F64 else "<i4"

    class _View:
        __cuda_array_interface__ = dict(shape=(int(n),), typestr=typestr, data=(int(ptr), False), version=2)
    return torch.as_tensor(_View(), device="cuda")


def allreduce_tensor(t, op: int, group=None):
    """In-place all-reduce of a record tensor (NCCL for CUDA tensors, gloo
    for CPU tensors): float64 sums or int32 minima."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == SUM_F64 else dist.ReduceOp.MIN, group=group)
    return t


class Callback:
    """An hmm_allreduce_fn that views each record the library passes as a
    tensor and hands it to `reduce(tensor, op, stream)`.  `calls` lists the
    (n, op) of every call; an exception is kept in `error` and makes the
    library call fail."""

    def __init__(self, reduce, device: str = "cuda"):
        self.reduce = reduce
        self.device = device
        self.calls = []
        self.error = None
        self.fn = _lib.ALLREDUCE_FN(self._call)

    def _call(self, ptr, n, op, stream, user):
        try:
            self.calls.append((int(n), int(op)))
            self.reduce(device_view(ptr, n, op, self.device), int(op), stream)
            return 0
        except Exception:
            self.error = traceback.format_exc()
            return 1

    @property
    def address(self):
        return C.cast(self.fn, C.c_void_p)


def dist_reduce(group=None):
    """reduce(tensor, op, stream): torch.distributed.all_reduce over `group`
    ordered on the library's stream (the current stream for CPU tensors)."""
    def reduce(t, op, stream):
        import torch
        if t.is_cuda:
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                allreduce_tensor(t, op, group)
        else:
            allreduce_tensor(t, op, group)
    return reduce


class Exchange:
    """Installs a Callback as the all-reduce of one hmm_stats object (default:
    torch.distributed over `group`).  Keep the object alive while the stats
    object is used; close() removes the hook."""

    def __init__(self, stats, group=None, reduce=None):
        self.cb = Callback(reduce or dist_reduce(group))
        self._lib = stats.lib
        self._stats = stats
        _lib.check(stats.lib.hmm_stats_set_allreduce(stats.h, self.cb.address, None))

    @property
    def calls(self):
        return self.cb.calls

    @property
    def error(self):
        return self.cb.error

    def close(self):
        if self._stats is not None:
            self._lib.hmm_stats_set_allreduce(self._stats.h, None, None)
            self._stats = None


def records(stats) -> list[tuple[int, int, int]]:
    """(device pointer, length, op) of the records hmm_estep_stats reduces."""
    out = []
    for i in range(3):
        p, n, op = C.c_void_p(), C.c_int64(), C.c_int32()
        _lib.check(stats.lib.hmm_stats_record(stats.h, i, C.byref(p), C.byref(n), C.byref(op)))
        out.append((p.value or 0, n.value, op.value))
    return out


def fit_data_parallel(ctx, model, batch, n_iter: int, group=None, opts=None, stream=None):
    """n_iter Baum-Welch iterations on this rank's shard `batch` with the
    records combined across the ranks of `group` before every M-step.
    Returns the total log-likelihood of all ranks' sequences entering each
    iteration, per model: [n_iter][n_models]."""
    from . import Stats, estep_stats, mstep
    stats = Stats(ctx, model)
    ex = Exchange(stats, group)
    trace = []
    try:
        for _ in range(n_iter):
            estep_stats(ctx, model, batch, stats=stats, stream=stream)
            trace.append(canonical_loglik(stats, model))
            mstep(ctx, model, stats, batch=batch, opts=opts, stream=stream)
    finally:
        ex.close()
    if ex.error:
        raise RuntimeError(ex.error)
    return np.array(trace)


def canonical_loglik(stats, model) -> np.ndarray:
    """Per-model sums of log-likelihoods in the (combined) statistic record
    (entry 1 of each model's slice of record 0)."""
    import torch
    torch.cuda.synchronize()
    p, n, op = records(stats)[0]
    rec = device_view(p, n, op).view(model.n_models, -1)
    return rec[:, 1].cpu().numpy().copy()
