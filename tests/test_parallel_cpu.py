"""Data-parallel exchange on CPU with two gloo ranks.

The library combines its records through a caller-supplied all-reduce
callback (hmm_stats_set_allreduce); paper_2605_29208_gb300.parallel supplies
it as a ctypes function of the C signature hmm_allreduce_fn.  Here each rank
calls that function pointer the way the library does, on host records laid
out as the library lays them out: the float64 statistic record (a sum over
sequences), the int32 support keys (minimum key, complemented maximum key:
one MIN reduction for both) and the per-Newton-pass float64 sums.  The
combined records must equal the whole batch's; the shards must partition
the sequences.  (The same exchange on the library's own device records, for
all 17 families, is tests/test_gpu_parallel.py.)"""
import ctypes as C
import os
import socket

import numpy as np
import pytest

from paper_2605_29208_gb300.parallel import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _record(model_d, values, offsets, idx):
    """[n_seq, sum logL, gamma_1 sums, xi sums, (W, Wy, Wy^2) per state] from
    the oracle for the sequences idx."""
    from oracle import hmm_oracle as O
    m = O.Model(model_d["family"], model_d["pi"], model_d["A"], dict(model_d["params"]))
    N = len(model_d["pi"])
    ll, g1, xi, fam = 0.0, np.zeros(N), np.zeros((N, N)), np.zeros((N, 3))
    for s in idx:
        y = values[offsets[s]:offsets[s + 1]]
        fb = O.forward_backward(m, y)
        ll += fb["logL"]
        g1 += fb["gamma"][0]
        xi += fb["xi_sum"]
        W = fb["gamma"]
        fam += np.stack([W.sum(0), (W * y[:, None]).sum(0), (W * y[:, None] ** 2).sum(0)], 1)
    return np.concatenate([[len(idx), ll], g1, xi.ravel(), fam.ravel()])


def ordered_key(v):
    """int32 key of a float32 whose integer order is the float order (the
    library's support-key encoding)."""
    i = np.asarray(v, np.float32).view(np.int32).astype(np.int64)
    return np.where(i >= 0, i, i ^ 0x7FFFFFFF).astype(np.int32)


def unkey(k):
    k = np.asarray(k, np.int64)
    return np.where(k >= 0, k, k ^ 0x7FFFFFFF).astype(np.int32).view(np.float32)


def _support_keys(values, offsets, idx, n_states):
    """[n_states][2]: key of the minimum, complemented key of the maximum of
    the rows of the shard (empty shard: the identities key(+inf),
    ~key(-inf))."""
    out = np.empty((n_states, 2), np.int32)
    rows = np.concatenate([values[offsets[s]:offsets[s + 1]] for s in idx]) if len(idx) else np.zeros(0)
    for j in range(n_states):
        r = rows[j::n_states] if len(rows) else rows
        lo = np.float32(r.min()) if len(r) else np.float32(np.inf)
        hi = np.float32(r.max()) if len(r) else np.float32(-np.inf)
        out[j] = [ordered_key(lo), ~ordered_key(hi)]
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2605_29208_gb300 import _lib, parallel, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    models = synth.small_models("gauss", 3, 1, seed=5)
    values, offsets, mid = synth.make_batch(3, models, [40, 7, 1, 90, 33, 12, 64], [0] * 7)
    S = len(offsets) - 1
    lo, hi = shard(S, rank, world)
    cb = parallel.Callback(parallel.dist_reduce(), device="cpu")
    fn = C.cast(cb.address, _lib.ALLREDUCE_FN)
    rec = np.ascontiguousarray(_record(models[0], values, offsets, range(lo, hi)))
    keys = np.ascontiguousarray(_support_keys(values, offsets, range(lo, hi), 3))
    passes = [np.ascontiguousarray(np.arange(9, dtype=np.float64) * (rank + 1) + p) for p in range(3)]
    rc = [fn(rec.ctypes.data, rec.size, parallel.SUM_F64, None, None),
          fn(keys.ctypes.data, keys.size, parallel.MIN_I32, None, None)]
    rc += [fn(p.ctypes.data, p.size, parallel.SUM_F64, None, None) for p in passes]
    # a failing reduction is reported to the library as a nonzero code
    bad = parallel.Callback(lambda t, op, s: (_ for _ in ()).throw(ValueError("boom")), device="cpu")
    rc_bad = C.cast(bad.address, _lib.ALLREDUCE_FN)(rec.ctypes.data, 1, parallel.SUM_F64, None, None)
    if rank == 0:
        full = _record(models[0], values, offsets, range(S))
        full_keys = _support_keys(values, offsets, range(S), 3)
        q.put(dict(rec=rec.tolist(), full=full.tolist(), keys=keys.tolist(), full_keys=full_keys.tolist(),
                   passes=[p.tolist() for p in passes], rc=rc, rc_bad=rc_bad, bad_error=bad.error or "",
                   calls=cb.calls, world=world))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_partition_sequences():
    for n in (0, 1, 7, 100):
        for w in (1, 2, 3, 8):
            got = [shard(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1


def test_support_key_encoding_orders_like_floats():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(0, 1e3, 500), [0.0, np.inf, -np.inf, 1e-38, -1e-38]]).astype(np.float32)
    k = ordered_key(v)
    o = np.argsort(v, kind="stable")
    assert np.all(np.diff(k[o].astype(np.int64)) >= 0)
    np.testing.assert_array_equal(unkey(k)[v != 0], v[v != 0])
    # the complement reverses the order: min over ~key is the max
    assert unkey(~np.min(~k)) == v.max()


def test_two_rank_gloo_exchange_through_the_callback():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got["rc"] == [0] * 5
    assert got["rc_bad"] == 1 and "boom" in got["bad_error"]
    np.testing.assert_allclose(got["rec"], got["full"], rtol=1e-12, atol=1e-9)
    keys = np.array(got["keys"], np.int32)
    full_keys = np.array(got["full_keys"], np.int32)
    np.testing.assert_array_equal(keys, full_keys)
    np.testing.assert_array_equal(unkey(keys[:, 0]), unkey(full_keys[:, 0]))
    for p, sums in enumerate(got["passes"]):
        np.testing.assert_array_equal(sums, np.arange(9) * 3 + 2 * p)
    assert [c[1] for c in got["calls"]] == [0, 1, 0, 0, 0]
