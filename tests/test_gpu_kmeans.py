"""k-means++ / Lloyd on the device (hmm_kmeans) against the oracle's
reading, for several restarts at once: the same seeds (bit-exact picks
from the shared uniforms), the same pass counts and labels, and centres
within float64 rounding.  Labels may only differ at an observation whose
two nearest centres are equidistant to rounding; such an observation must
still be assigned to one of them."""
import numpy as np
import pytest

from oracle import hmm_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_29208_gb300 as H
    from paper_2605_29208_gb300 import build
    build.build()
    return H


@pytest.mark.parametrize("T,F,K,R", [(1, 1, 1, 1), (997, 1, 3, 4), (5000, 2, 8, 3), (40000, 3, 5, 2),
                                     (3000, 16, 64, 1)])
def test_kmeans_matches_oracle(H, T, F, K, R):
    rng = np.random.default_rng(T + F + K)
    X = (rng.normal(0, 1, (T, F)) + 3.0 * rng.integers(0, max(K, 1), T)[:, None]).astype(np.float32)
    u = rng.random((R, K))
    ctx = H.Context(0)
    C, lab, passes = H.kmeans(ctx, X, u, max_iter=100)
    C, lab = C.cpu().numpy(), lab.cpu().numpy()
    X64 = X.astype(np.float64)
    for r in range(R):
        Cr, lr, pr = O.kmeanspp(X64, u[r], max_iter=100)
        # the seeds alone (no Lloyd pass) are picked bit for bit
        C0, _, _ = O.kmeanspp(X64, u[r], max_iter=0)
        S0, _, _ = H.kmeans(ctx, X, u[r:r + 1], max_iter=0)
        np.testing.assert_array_equal(S0.cpu().numpy()[0], C0)
        assert passes[r] == pr
        np.testing.assert_allclose(C[r], Cr, rtol=1e-12, atol=1e-12)
        diff = np.nonzero(lab[r] != lr)[0]
        for i in diff:
            d = np.sum((X64[i] - Cr) ** 2, axis=1)
            assert abs(d[lab[r][i]] - d.min()) <= 1e-12 * max(1.0, d.min())


def test_kmeans_rejects_bad_arguments(H):
    ctx = H.Context(0)
    from paper_2605_29208_gb300 import HmmError
    X = np.zeros((10, 1), np.float32)
    with pytest.raises(HmmError):
        H.kmeans(ctx, X, np.array([[0.5, 1.0]]))          # a uniform outside [0, 1)
    with pytest.raises(HmmError):
        H.kmeans(ctx, X, np.full((1, 65), 0.5))           # more than 64 clusters


def test_device_restarts_start_like_the_host_reading(H):
    """initialize.kmeanspp_init on the device and on the host give the same
    starting model (same uniforms, same rules)."""
    from paper_2605_29208_gb300 import initialize, synth
    truth, values, offsets, mid = synth.tiny_gauss()
    ctx = H.Context(0)
    for seed in (0, 1, 2):
        a = initialize.kmeanspp_init("gauss", 2, values, offsets, seed=seed)
        b = initialize.kmeanspp_init("gauss", 2, values, offsets, seed=seed, ctx=ctx)
        np.testing.assert_allclose(b["A"], a["A"], rtol=1e-12)
        for k in a["params"]:
            np.testing.assert_allclose(b["params"][k], a["params"][k], rtol=1e-10, atol=1e-12)
