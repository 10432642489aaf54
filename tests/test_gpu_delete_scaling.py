"""Delete latency stays flat as the window grows (the paper's O(1) delete,
Sec. 3.5.2: the address-translation table gives each id its slab and slot
directly, so a batch of B deletes touches B table entries and B slabs
whatever the window's size).  One index of the serving workload's vectors
(d=128, nlist=16384, slab 128) is grown from 1,000,000 to 10,000,000 live
vectors; at each size sliding-window steps insert 10,000 new vectors and
delete the 10,000 oldest, and the delete's device time (CUDA events on its
stream) is compared: the median at 10 M stays within 1.5x of the median at
1 M.  The state after the steps is checked for the counts the steps
imply."""
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


def test_delete_time_flat_from_1m_to_10m(torch):
    from paper_2601_11808_gb300.sivf import Index
    w = W.CONFIGS["serving"]
    top, B, steps = 10_000_000, 10_000, 40
    n_max = top + (1 << 20)
    S = int(1.02 * top / w.slab_size) + 3 * w.nlist + (1 << 12)
    ctr = W.centers(w)
    pool = W.noise_pool(w, 1 << 18)
    g = Index(w.d, w.nlist, w.slab_size, n_max, S)
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).cuda())
    ctr_d, pool_d = torch.from_numpy(ctr).cuda(), torch.from_numpy(pool).cuda()
    sig = float(np.float32(w.sigma))
    stream = torch.cuda.current_stream()

    def add_range(b, n):
        for c0 in range(b, b + n, 2_000_000):
            m = min(2_000_000, b + n - c0)
            c, r = W.pooled_parts(w, c0, m, len(pool))
            x = ctr_d[torch.from_numpy(c).cuda()] + pool_d[torch.from_numpy(r).cuda()] * sig
            g.add(torch.from_numpy(W.stream_ids(c0, m, n_max)).cuda(), x)

    lo = hi = 0
    med = {}
    for Wn in (1_000_000, top):
        add_range(hi, Wn - (hi - lo))
        hi = lo + Wn
        g.sync()
        ms = []
        for st in range(steps + 3):
            add_range(hi, B)
            hi += B
            ids = torch.from_numpy(W.stream_ids(lo, B, n_max)).cuda()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.remove(ids)
            e1.record(stream)
            lo += B
            e1.synchronize()
            if st >= 3:
                ms.append(e0.elapsed_time(e1))
        assert g.sync() == B                      # the last delete removed all B
        assert g.stats()["ntotal"] == Wn
        med[Wn] = float(np.median(ms))
    g.close()
    assert med[top] <= 1.5 * med[1_000_000], med
