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
    # the regular search of the same shape loads the kernels both paths
    # share (so lazy module loading cannot show up as memory taken below)
    g.search(q, 10, 8)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()       # a stream neither search has used
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(stream):
        for _ in range(3):             # the first call on the stream included
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


def _need_bytes(nq, P, k, L, tq, ips, rows):
    """The allocation-free search's scratch bytes for a plan (the same sum,
    each part rounded up to 256 bytes, as the library's carve-up)."""
    run_cap = nq * P + 2 * tq * ips * 152
    item_cap = nq * P + L + ips * 152
    parts = [64, nq * P * 4, L * 4, (L + 1) * 4, (L + 1) * 4, L * 4, nq * P * 4, nq * P * 4,
             run_cap * k * 4, run_cap * k * 8, nq * 4, nq * P * 4, nq * 16, item_cap * 8,
             rows * L * 4]
    b = 0
    for n in parts:
        b = ((b + 255) & ~255) + n
    return b


def test_noalloc_narrows_a_plan_that_does_not_fit(torch):
    """A batch whose default plan needs more than the fixed array but fits
    once the work items per SM are lowered: the call narrows the plan
    (items per SM, then coarse rows) and still returns sivf_search's
    results."""
    from paper_2601_11808_gb300 import sivf
    w = W.CONFIGS["tiny_window"]
    g, ctr = _index(torch, w, 20_000)
    nq, k, P = 3000, 48, 8
    t = g.get_tile("fp32", nq, k, P)
    cap = 32 << 20
    rows = min(nq, max(1, (8 << 20) // (4 * w.nlist)))
    ips = t["items_per_sm"]
    assert _need_bytes(nq, P, k, w.nlist, t["queries_per_tile"], ips, rows) > cap
    while _need_bytes(nq, P, k, w.nlist, t["queries_per_tile"], ips, rows) > cap and ips > 1:
        ips >>= 1
    while _need_bytes(nq, P, k, w.nlist, t["queries_per_tile"], ips, rows) > cap and rows > 1:
        rows >>= 1
    assert ips < t["items_per_sm"]
    assert _need_bytes(nq, P, k, w.nlist, t["queries_per_tile"], ips, rows) <= cap
    q = W.queries(w, 0, nq, ctr)
    for _ in range(2):
        compare_topk(*_both(torch, g, q, k, P), RTOL, "noalloc narrowed plan")
