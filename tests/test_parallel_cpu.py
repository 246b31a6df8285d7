"""Data-parallel Baum-Welch exchange on CPU: two gloo ranks each compute the
statistic record of their shard of sequences; the element-wise all-reduce
must equal the record of the whole batch (the one exchange step of an
iteration), and the shards must partition the sequences."""
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


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_2605_29208_gb300 import synth
    from paper_2605_29208_gb300.parallel import allreduce_stats
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    models = synth.small_models("gauss", 3, 1, seed=5)
    values, offsets, mid = synth.make_batch(3, models, [40, 7, 1, 90, 33, 12, 64], [0] * 7)
    lo, hi = shard(len(offsets) - 1, rank, world)
    rec = torch.from_numpy(_record(models[0], values, offsets, range(lo, hi)))
    allreduce_stats(rec)
    if rank == 0:
        full = _record(models[0], values, offsets, range(len(offsets) - 1))
        q.put((rec.numpy().tolist(), full.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_partition_sequences():
    for n in (0, 1, 7, 100):
        for w in (1, 2, 3, 8):
            got = [shard(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1


def test_two_rank_gloo_allreduce_equals_full_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, full = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    np.testing.assert_allclose(got, full, rtol=1e-12, atol=1e-9)
