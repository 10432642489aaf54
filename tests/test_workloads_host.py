"""Host logic of the batch schedules, request streams, pooled-noise windows
and the tile-bucket rule (no GPU)."""
import math

import numpy as np

from paper_2601_11808_gb300 import workloads as W
from paper_2601_11808_gb300 import autotune


def test_mixed_schedule_shape():
    s = W.mixed_schedule(64, 4096, 100_000, 50_000, (8, 16, 32, 64, 128), seed=0)
    assert len(s) == 192
    assert [k for k, _, _ in s[:6]] == ["add", "remove", "search"] * 2
    for kind, n, p in s:
        hi = {"add": 50_000, "remove": 100_000, "search": 4096}[kind]
        assert 1 <= n <= hi
        assert (p in (8, 16, 32, 64, 128)) == (kind == "search")
    # log-uniform: about half the sizes below sqrt(hi)
    q = np.asarray([n for k, n, _ in s if k == "search"])
    assert 0.25 < np.mean(q < 64) < 0.75
    assert s == W.mixed_schedule(64, 4096, 100_000, 50_000, (8, 16, 32, 64, 128), seed=0)


def test_request_stream_statistics():
    t, kind, size = W.request_stream(20000, 4000.0, seed=1)
    assert (np.diff(t) >= 0).all()
    assert abs(t[-1] / 1e9 - 20000 / 4000.0) < 0.3            # Poisson rate
    frac = np.bincount(kind, minlength=3) / len(kind)
    np.testing.assert_allclose(frac, [0.7, 0.1, 0.2], atol=0.02)
    assert size[kind == 2].max() <= 256 and size.min() >= 1
    assert size[kind == 0].max() <= 10_000


def test_pooled_window_is_positional():
    w = W.CONFIGS["serving"]
    ctr = W.centers(w)
    pool = W.noise_pool(w, 1 << 12)
    a = W.pooled_vectors(w, 4000, 300, ctr, pool)
    b = W.pooled_vectors(w, 3900, 500, ctr, pool)[100:400]
    np.testing.assert_array_equal(a, b)
    c, r = W.pooled_parts(w, 4000, 300, len(pool))
    exp = (ctr[c] + pool[r] * np.float32(w.sigma)).astype(np.float32)
    np.testing.assert_array_equal(a, exp)
    assert a.dtype == np.float32 and c.max() < w.n_comp and r.max() < len(pool)


def test_bucket_rule():
    # pairs per list nq * nprobe / nlist, log2 floor, offset 8, clamped to [0, 23]
    for nq, P, L in [(1, 1, 16384), (10000, 8, 1024), (40, 8, 64), (1 << 20, 1024, 1)]:
        r = max(nq * P / L, 1 / 256)
        b = min(max(math.floor(math.log2(r)) + 8, 0), 23)
        assert autotune.bucket(L, nq, 10, P, "fp32") == f"fp32/{b}/0"
    assert autotune.bucket(64, 40, 10, 8, "bf16").endswith("/1")    # 4k = 40 kept
    assert autotune.bucket(64, 40, 100, 8, "bf16").endswith("/3")   # 400 kept


def test_zipf_law_and_draws():
    """The skewed mixture: P(rank r) = r^-s / H(n, s); the rank -> component
    map is a fixed permutation; empirical component shares follow the law;
    vectors stay positional (independent of batching)."""
    w = W.small("tiny_window", n_comp=32, zipf=1.0)
    p, perm = W.zipf_law(w)
    h = sum(1.0 / r for r in range(1, 33))
    np.testing.assert_allclose(p, [1.0 / (r * h) for r in range(1, 33)], rtol=1e-12)
    assert sorted(perm.tolist()) == list(range(32))
    np.testing.assert_array_equal(perm, W.zipf_law(w)[1])
    ctr = W.centers(w)
    x = W.vectors(w, 0, 40_000, ctr)
    # nearest center of each vector (sigma 0.1 against centers in [-1, 1]^32:
    # the component that drew it)
    d2 = ((x[:, None, :] - ctr[None, :, :]) ** 2).sum(-1)
    share = np.bincount(d2.argmin(1), minlength=32) / len(x)
    for rank in (1, 2, 4, 8):
        assert abs(share[perm[rank - 1]] - p[rank - 1]) < 4 * math.sqrt(p[rank - 1] / len(x)) + 1e-3
    np.testing.assert_array_equal(W.vectors(w, 1000, 5000, ctr), x[1000:6000])
    # zipf = 0 is the uniform mixture
    u = W.small("tiny_window", zipf=0.0)
    np.testing.assert_array_equal(W.vectors(u, 0, 100), W.vectors(W.CONFIGS["tiny_window"], 0, 100))
