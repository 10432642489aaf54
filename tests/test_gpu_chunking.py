"""Query chunks of a search: a batch whose scratch exceeds the chunk budget
is searched in chunks of queries, each chunk streaming the lists its queries
probe.  The answer of a query does not depend on the other queries of its
chunk (each candidate stage keeps the exact best K' by (distance, slot), the
re-rank and the FP32 scan are per query), so a search cut into chunks of 256
queries (budget 1 byte: the smallest chunk) returns the same distances and
ids, bit for bit, as the same search in one chunk, in every scan form, with
one probe and with several, and with a ragged last chunk."""
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


def test_chunked_search_equals_one_chunk(torch):
    from paper_2601_11808_gb300 import sivf
    w = W.small("sift_window", n_comp=64, nlist=64, slab_size=64)
    ctr = W.centers(w)
    n = 30_000
    g = sivf.Index(w.d, w.nlist, w.slab_size, 2 * n, 2 * (n // w.slab_size + w.nlist), 0,
                   ("bf16", "fp8"))
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).cuda())
    g.add(torch.from_numpy(W.stream_ids(0, n, 2 * n)).cuda(),
          torch.from_numpy(W.vectors(w, 0, n, ctr)).cuda(), sync=True)
    q = torch.from_numpy(W.queries(w, 0, 1500, ctr)).cuda()   # 5 chunks of 256 + 220
    for form, k, P in (("fp32", 10, 1), ("fp32", 10, 6), ("bf16", 10, 1), ("bf16", 25, 6),
                       ("fp8", 10, 1), ("fp8", 10, 6)):
        sivf.sivf_set_chunk_bytes(g.h, 0)
        d1, i1 = g.search(q, k, P, form)
        sivf.sivf_set_chunk_bytes(g.h, 1)
        d2, i2 = g.search(q, k, P, form)
        np.testing.assert_array_equal(i1.cpu().numpy(), i2.cpu().numpy(), err_msg=f"{form} P{P}")
        np.testing.assert_array_equal(d1.cpu().numpy(), d2.cpu().numpy(), err_msg=f"{form} P{P}")
    sivf.sivf_set_chunk_bytes(g.h, 0)
    with pytest.raises(sivf.SivfError):
        sivf.sivf_set_chunk_bytes(g.h, -1)
    g.close()
