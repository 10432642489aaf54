"""GPU parity of coarse-quantizer training (Lloyd's k-means, sivf_train)
against the oracle's k-means.

- Quantized training rows (multiples of 2^-6 in [-2, 2]): every FP64 sum is
  exact, so the order of the device's atomic additions cannot matter and the
  centroids must equal the oracle's bit for bit, with the same final
  assignment.
- General float rows: centroids equal within 2 units in the last place
  (FP64 sums in another order), and the trained index then matches the
  oracle built on the same centroids.
- Errors: fewer rows than lists; training a non-empty index.
"""
import numpy as np
import pytest

import oracle
from sivf_check import build_lib
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def _index(torch, d, L, n_max=20000):
    from paper_2601_11808_gb300.sivf import Index
    return Index(d, L, 32, n_max, 4 * (n_max // 32 + L))


@pytest.mark.parametrize("d,L,iters,seed", [(32, 64, 4, 3), (16, 40, 6, 11), (128, 96, 3, 5)])
def test_train_bit_exact_on_quantized_rows(torch, d, L, iters, seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(-96, 97, (L, d))
    x = (ctr[rng.integers(0, L, 6000)] + rng.integers(-8, 9, (6000, d))) / 64.0
    x = x.astype(np.float32)
    g = _index(torch, d, L)
    g.train(torch.from_numpy(x).cuda(), iters, seed)
    c_gpu = g.centroids().cpu().numpy()
    c_ora, lab_ora = oracle.kmeans(x, L, iters, seed)
    np.testing.assert_array_equal(c_gpu, c_ora)
    np.testing.assert_array_equal(g.assign(torch.from_numpy(x).cuda()).cpu().numpy(), lab_ora)


def test_train_float_rows_then_index_parity(torch):
    w = W.CONFIGS["tiny_window"]
    ctr = W.centers(w)
    x = W.vectors(w, 0, 8000, ctr)
    g = _index(torch, w.d, w.nlist)
    g.train(torch.from_numpy(x).cuda(), 3, 7)
    c_gpu = g.centroids().cpu().numpy()
    c_ora, _ = oracle.kmeans(x, w.nlist, 3, 7)
    np.testing.assert_array_max_ulp(c_gpu, c_ora, maxulp=2)
    # the trained index stores and finds like the oracle on its centroids
    o = oracle.OracleIVF(w.d, w.nlist, 32, 20000, 4 * (20000 // 32 + w.nlist))
    o.set_centroids(c_gpu)
    ids = np.arange(8000, dtype=np.int64)
    g.add(torch.from_numpy(ids).cuda(), torch.from_numpy(x).cuda())
    o.add(ids, x)
    q = W.queries(w, 0, 50, ctr)
    gd, gi = g.search(torch.from_numpy(q).cuda(), 10, 8)
    od, oi = o.search(q, 10, 8)
    np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=1e-5)
    assert np.mean([set(a) == set(b) for a, b in zip(gi.cpu().numpy().tolist(), oi.tolist())]) >= 0.99


def test_train_errors(torch):
    from paper_2601_11808_gb300.sivf import SivfError
    x = np.random.default_rng(0).standard_normal((100, 16)).astype(np.float32)
    g = _index(torch, 16, 200)
    with pytest.raises(SivfError):
        g.train(torch.from_numpy(x).cuda(), 2, 0)          # n < nlist
    g = _index(torch, 16, 10)
    g.train(torch.from_numpy(x).cuda(), 2, 0)
    g.add(torch.arange(5, dtype=torch.int64).cuda(), torch.from_numpy(x[:5]).cuda())
    with pytest.raises(SivfError):
        g.train(torch.from_numpy(x).cuda(), 2, 0)          # not empty
