"""The allocation-free forward-backward entry point (hmm_forward_backward_static).

Some callers cannot allocate device memory at the moment they ask for a
posterior: code inside a memory pool that must not be bypassed, a
latency-bound loop that cannot take cudaMalloc's implicit synchronisation,
or a process that has already claimed the free memory.  The entry point runs
the forward-backward with its scratch in a fixed array inside the library.

These tests check that it gives the same log-likelihoods and occupancies as
hmm_forward_backward and as the float64 oracle on two calls in a row (the
shared scratch keeps the previous call's contents, so the second call also
checks that nothing stale leaks through), that it really makes no device
allocation, that an oversized batch is refused, and that a malformed batch
is caught on the device without touching memory outside the caller's
buffers.  The file runs last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

from oracle import hmm_oracle as O
from paper_2605_29208_gb300 import synth

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


def om(d):
    return O.Model(d["family"], d["pi"].copy(), d["A"].copy(), {k: np.array(v, copy=True) for k, v in d["params"].items()})


def test_static_scratch_forward_backward_matches_allocating_call(H):
    import torch
    ctx = H.Context(0)
    models = synth.small_models("gamma", 5, 2, seed=91)
    lengths = [1, 2, 0, 9, 130, 777, 64, 3]
    mid = np.arange(len(lengths)) % 2
    values, offsets, mid = synth.make_batch(17, models, lengths, mid)
    model = H.Model(ctx, models)
    batch = H.Batch(values, offsets, mid)
    ref_ll, ref_g, _ = H.forward_backward(ctx, model, batch)
    ref_ll = ref_ll.cpu().numpy()
    ref_g = ref_g.cpu().numpy()
    # a second, larger batch first, so the scratch holds unrelated data
    v2, o2, m2 = synth.make_batch(18, models, [1500, 900], [0, 1])
    b2 = H.Batch(v2, o2, m2)
    H.forward_backward_static(model, b2, torch.empty((b2.total_T, model.N), device="cuda"),
                              torch.empty(b2.n_seq, dtype=torch.float64, device="cuda"))
    for _ in range(2):
        gamma = torch.full((batch.total_T, model.N), float("nan"), device="cuda")
        ll = torch.full((batch.n_seq,), float("nan"), dtype=torch.float64, device="cuda")
        H.forward_backward_static(model, batch, gamma, ll)
        torch.cuda.synchronize()
        got_ll = ll.cpu().numpy()
        got_g = gamma.cpu().numpy()
        np.testing.assert_allclose(got_ll, ref_ll, rtol=LL_RTOL, atol=LL_RTOL)
        np.testing.assert_allclose(got_g, ref_g, atol=GAMMA_ATOL, rtol=0)
        # and against the float64 oracle, sequence by sequence
        for s in range(len(lengths)):
            y = values[offsets[s]:offsets[s + 1]]
            if len(y) == 0:
                assert got_ll[s] == 0.0
                continue
            fb = O.forward_backward(om(models[mid[s]]), y)
            assert abs(got_ll[s] - fb["logL"]) <= LL_RTOL * max(1.0, abs(fb["logL"]))
            np.testing.assert_allclose(got_g[offsets[s]:offsets[s + 1]], fb["gamma"], atol=GAMMA_ATOL, rtol=0)
    assert ctx.status() == 0


def test_static_call_allocates_no_device_memory(H):
    """After a warm-up call (which loads the kernels), a call on a larger
    batch with the same sequence count leaves the device's free memory
    unchanged: the scratch is the library's fixed array."""
    import torch
    ctx = H.Context(0)
    models = synth.small_models("gauss", 8, 1, seed=5)
    model = H.Model(ctx, models)
    v1, o1, m1 = synth.make_batch(21, models, [100] * 64, [0] * 64)
    v2, o2, m2 = synth.make_batch(22, models, [4000] * 64, [0] * 64)
    b1, b2 = H.Batch(v1, o1, m1), H.Batch(v2, o2, m2)
    outs = [(torch.empty((b.total_T, model.N), device="cuda"),
             torch.empty(b.n_seq, dtype=torch.float64, device="cuda")) for b in (b1, b2)]
    H.forward_backward_static(model, b1, *outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    H.forward_backward_static(model, b2, *outs[1])
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    ll = outs[1][1].cpu().numpy()
    s = 7
    fb = O.forward_backward(om(models[0]), v2[o2[s]:o2[s + 1]])
    assert abs(ll[s] - fb["logL"]) <= LL_RTOL * abs(fb["logL"])


def test_static_scratch_rejects_oversized_batch(H):
    import torch
    ctx = H.Context(0)
    models = synth.small_models("gauss", 16, 1, seed=3)
    model = H.Model(ctx, models)
    total = (32 << 20) // (16 * 4) + 10           # just past the 32 MiB limit
    offsets = np.array([0, total], np.int64)
    batch = H.Batch(np.zeros(total), offsets, np.zeros(1, np.int32))
    with pytest.raises(H.HmmError) as e:
        H.forward_backward_static(model, batch, torch.empty((total, 16), device="cuda"),
                                  torch.empty(1, dtype=torch.float64, device="cuda"))
    assert "scratch" in str(e.value)


@pytest.mark.parametrize("case", ["decreasing_offsets", "last_offset", "model_id"])
def test_static_call_rejects_malformed_batch_on_device(H, case):
    """Offsets and model ids are device data: the call checks them on the
    device, runs no sequence, writes NaN log-likelihoods, leaves the
    occupancy buffer untouched and reports HMM_E_ARG through the context's
    sticky status."""
    import torch
    ctx = H.Context(0)
    models = synth.small_models("gauss", 4, 2, seed=8)
    model = H.Model(ctx, models)
    offsets = np.array([0, 50, 80, 120], np.int64)
    mid = np.array([0, 1, 0], np.int32)
    total = 120
    dev_offsets = offsets.copy()
    if case == "decreasing_offsets":
        dev_offsets[2] = 20
    elif case == "last_offset":
        dev_offsets[3] = 119
    else:
        mid = np.array([0, 2, 0], np.int32)
    batch = H.Batch(np.ones(total), offsets, mid)
    batch.offsets.copy_(torch.as_tensor(dev_offsets))
    gamma = torch.full((total, model.N), 7.0, device="cuda")
    ll = torch.zeros(3, dtype=torch.float64, device="cuda")
    H.forward_backward_static(model, batch, gamma, ll)
    assert ctx.status() == 1                       # HMM_E_ARG
    assert np.all(np.isnan(ll.cpu().numpy()))
    assert bool((gamma == 7.0).all())
    # a well-formed call afterwards works again
    batch.offsets.copy_(torch.as_tensor(offsets))
    batch.model_id.copy_(torch.as_tensor(np.array([0, 1, 0], np.int32)))
    H.forward_backward_static(model, batch, gamma, ll)
    assert ctx.status() == 0
    assert np.all(np.isfinite(ll.cpu().numpy()))
