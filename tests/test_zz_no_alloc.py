"""The allocation-free search (sivf_search_noalloc) against the regular one.

Callers such as a serving process whose memory pool owns the whole GPU, or
a latency-critical loop that must not enter the allocator, cannot let the
library cudaMalloc during a call.  sivf_search_noalloc takes its scratch
from a fixed array in the library's device code instead.  These tests call
it through the C ABI and check, on two calls in a row (and again after
another index used the same array), that it returns what sivf_search
returns, within the tolerance of the other search tests.  This file is
collected last so that a run stopping at its first failure has run every
other test before it.
"""
import numpy as np
import pytest

from sivf_check import build_lib, compare_topk
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def _index(torch, w, n, seed_shift=0):
    from paper_2601_11808_gb300 import sivf
    ctr = W.centers(w)
    n_max = 2 * n
    g = sivf.Index(w.d, w.nlist, w.slab_size, n_max, 2 * (n // w.slab_size + w.nlist))
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).cuda())
    x = W.vectors(w, seed_shift, n, ctr)
    g.add(torch.from_numpy(W.stream_ids(0, n, n_max)).cuda(), torch.from_numpy(x).cuda())
    g.sync()
    return g, ctr


def _both(torch, g, q, k, P):
    from paper_2601_11808_gb300 import sivf
    qd = torch.from_numpy(q).cuda()
    d0, i0 = g.search(qd, k, P)
    d1 = torch.full((q.shape[0], k), -1.0, dtype=torch.float32, device="cuda")
    i1 = torch.full((q.shape[0], k), -7, dtype=torch.int64, device="cuda")
    sivf.sivf_search_noalloc(g.h, qd, k, P, d1, i1)
    torch.cuda.synchronize()
    return (d1.cpu().numpy(), i1.cpu().numpy(), d0.cpu().numpy().astype(np.float64),
            i0.cpu().numpy())


def test_noalloc_search_matches_search_on_consecutive_calls(torch):
    w = W.CONFIGS["tiny_window"]
    g, ctr = _index(torch, w, 20_000)
    qa = W.queries(w, 0, 200, ctr)
    qb = W.queries(w, 200, 333, ctr)
    for q, k, P in ((qa, 10, 8), (qb, 17, 3), (qa, 10, 8)):
        compare_topk(*_both(torch, g, q, k, P), RTOL, f"noalloc k{k} P{P}")
    # a second index of another shape uses the same array in between
    w2 = W.small("tiny_window", nlist=48, slab_size=64)
    g2, ctr2 = _index(torch, w2, 9_000)
    q2 = W.queries(w2, 0, 150, ctr2)
    compare_topk(*_both(torch, g2, q2, 5, 48), RTOL, "noalloc second index")
    compare_topk(*_both(torch, g, qb, 10, 8), RTOL, "noalloc first index again")


def test_noalloc_does_not_allocate_and_refuses_oversize(torch):
    from paper_2601_11808_gb300 import sivf
    w = W.CONFIGS["tiny_window"]
    g, ctr = _index(torch, w, 5_000)
    q = torch.from_numpy(W.queries(w, 0, 64, ctr)).cuda()
    d = torch.empty((64, 10), dtype=torch.float32, device="cuda")
    i = torch.empty((64, 10), dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()       # a stream sivf_search never used
    with torch.cuda.stream(stream):
        sivf.sivf_search_noalloc(g.h, q, 10, 8, d, i)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            sivf.sivf_search_noalloc(g.h, q, 10, 8, d, i)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    big = torch.zeros((20_000, w.d), dtype=torch.float32, device="cuda")
    bd = torch.empty((20_000, 64), dtype=torch.float32, device="cuda")
    bi = torch.empty((20_000, 64), dtype=torch.int64, device="cuda")
    with pytest.raises(sivf.SivfError) as e:
        sivf.sivf_search_noalloc(g.h, big, 64, 64, bd, bi)
    assert e.value.status == sivf.E_ARG and "scratch" in str(e.value)
