"""The allocation-free forward-backward entry point (hmm_forward_backward_static)
gives the same log-likelihoods and occupancies as hmm_forward_backward, on
two calls in a row (the shared scratch array keeps the previous call's
contents, so the second call checks that nothing stale leaks through).

It is meant for callers that must not allocate device memory during the
call (a pool they do not control, a latency-bound loop); this file runs
last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_2605_29208_gb300 import synth

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
GAMMA_ATOL = 1e-4


def test_static_scratch_forward_backward_matches_allocating_call():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
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


def test_static_scratch_rejects_oversized_batch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
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
