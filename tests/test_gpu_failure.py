"""Failure paths of the index, exercised without any device fault.

The paper's fail-fast rule (Sec. 3.2) and its bounded traversal (Sec. 3.3):
a device-side bound, or a device wait that runs out, records a sticky error;
the next synchronising call reports it and every later call refuses work
without enqueuing anything.  Both injections here are safe for the GPU:

- a sticky error bit written into the index's device error word from the
  host (the test hook sivf_debug_set_error_bits), as a corrupt directory
  walk would leave it;
- a wait limit of 1 ns for the list scan (sivf_set_wait_limit): a wait of
  the tensor-core scan then really runs out, the scan's roles stop (the
  copies already in flight are drained first, under the default limit) and
  the status comes back as a timeout.
"""
import numpy as np
import pytest

from sivf_check import build_lib
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def _index(torch, n=4000):
    from paper_2601_11808_gb300.sivf import Index
    w = W.small("tiny_window", nlist=32, slab_size=32)
    ctr = W.centers(w)
    n_max = 2 * n
    g = Index(w.d, w.nlist, w.slab_size, n_max, 2 * (n // w.slab_size + w.nlist), 0,
              ("bf16", "fp8"))
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).cuda())
    x = W.vectors(w, 0, n, ctr)
    g.add(torch.from_numpy(W.stream_ids(0, n, n_max)).cuda(), torch.from_numpy(x).cuda(),
          sync=True)
    return w, g, ctr


def _same_dump(a, b):
    for key in a:
        if isinstance(a[key], np.ndarray):
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)
        else:
            assert a[key] == b[key], key


def _refused(call, statuses):
    from paper_2601_11808_gb300.sivf import SivfError
    with pytest.raises(SivfError) as e:
        call()
    assert e.value.status in statuses, (e.value.status, str(e.value))


def _every_call_refused(torch, w, g, ctr, statuses):
    from paper_2601_11808_gb300 import sivf
    q = torch.from_numpy(W.queries(w, 0, 8, ctr)).cuda()
    x = torch.from_numpy(W.vectors(w, 10_000, 40, ctr)).cuda()   # >= nlist rows (train)
    ids = torch.arange(6000, 6040, dtype=torch.int64, device="cuda")
    d = torch.empty((8, 5), dtype=torch.float32, device="cuda")
    i = torch.empty((8, 5), dtype=torch.int64, device="cuda")
    before = g.dump()
    _refused(lambda: g.add(ids, x, sync=True), statuses)
    _refused(lambda: g.remove(ids[:4], sync=True), statuses)
    for form in ("fp32", "bf16", "fp8"):
        _refused(lambda: g.search(q, 5, 4, form), statuses)
    _refused(lambda: sivf.sivf_search_noalloc(g.h, q, 5, 4, d, i), statuses)
    _refused(lambda: g.compact(1, 1 << 40, sync=True), statuses)
    _refused(lambda: g.train(x, 1, 0), statuses)
    _refused(lambda: g.executor([{"kind": "search", "q": q, "k": 5, "nprobe": 4,
                                  "dtype": "fp32", "dist": d, "labels": i}]), statuses)
    _refused(lambda: sivf.Server(g, k=5, nprobe=4), statuses)
    torch.cuda.synchronize()
    _same_dump(before, g.dump())


def test_sticky_error_bit_is_reported_then_every_call_refused(torch):
    from paper_2601_11808_gb300 import sivf
    w, g, ctr = _index(torch)
    q = torch.from_numpy(W.queries(w, 0, 8, ctr)).cuda()
    g.search(q, 5, 4, "bf16")                        # a healthy call first
    sivf.sivf_debug_set_error_bits(g.h, 1)           # a bad slab reference
    _refused(lambda: g.sync(), (sivf.E_CORRUPT,))
    assert g.stats()["error_bits"] == 1
    _every_call_refused(torch, w, g, ctr, (sivf.E_CORRUPT,))
    g.close()


def test_timeout_bit_reports_timeout(torch):
    from paper_2601_11808_gb300 import sivf
    w, g, ctr = _index(torch, 2000)
    sivf.sivf_debug_set_error_bits(g.h, 8)
    _refused(lambda: g.sync(), (sivf.E_TIMEOUT,))
    _every_call_refused(torch, w, g, ctr, (sivf.E_CORRUPT, sivf.E_TIMEOUT))
    g.close()


@pytest.mark.parametrize("form", ["bf16", "fp8"])
def test_scan_wait_that_runs_out_is_reported_as_timeout(torch, form):
    """With a 1 ns limit the first wait of the tensor-core scan that is not
    already satisfied (a TMA copy landing, an MMA finishing) gives up: the
    scan stops and the sticky timeout bit comes back through sivf_sync; the
    GPU context stays usable (another index on the same device searches
    normally afterwards, also under the default limit)."""
    from paper_2601_11808_gb300 import sivf
    w, g, ctr = _index(torch)
    q = torch.from_numpy(W.queries(w, 0, 64, ctr)).cuda()
    ref_d, ref_i = g.search(q, 5, 4, form)
    torch.cuda.synchronize()
    sivf.sivf_set_wait_limit(g.h, 1)
    g.search(q, 5, 4, form)
    _refused(lambda: g.sync(), (sivf.E_TIMEOUT,))
    assert g.stats()["error_bits"] & 8
    _every_call_refused(torch, w, g, ctr, (sivf.E_CORRUPT, sivf.E_TIMEOUT))
    g.close()
    # the context is intact: a fresh index gives the same answers as before
    w2, g2, ctr2 = _index(torch)
    d2, i2 = g2.search(q, 5, 4, form)
    np.testing.assert_array_equal(i2.cpu().numpy(), ref_i.cpu().numpy())
    np.testing.assert_array_equal(d2.cpu().numpy(), ref_d.cpu().numpy())
    g2.close()


def test_wait_limit_arguments(torch):
    from paper_2601_11808_gb300 import sivf
    w, g, ctr = _index(torch, 1000)
    _refused(lambda: sivf.sivf_set_wait_limit(g.h, -1), (sivf.E_ARG,))
    sivf.sivf_set_wait_limit(g.h, 0)                 # back to the default
    q = torch.from_numpy(W.queries(w, 0, 8, ctr)).cuda()
    g.search(q, 5, 4, "bf16")
    g.sync()
    g.close()
