"""Checkpoint of the device state (sivf_save / sivf_load): the loaded index
equals the saved one array for array and searches identically in every scan
form; after the same further batches both match the oracle's logical state
and return the same results.  A missing or foreign file is refused."""
import os

import numpy as np
import pytest

import oracle
from sivf_check import build_lib, compare_state
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def _payload_equal(a, b):
    pa = a.dump_payload(bf16=True, fp8=True)
    pb = b.dump_payload(bf16=True, fp8=True)
    for k in pa:
        np.testing.assert_array_equal(pa[k], pb[k], err_msg=k)


def _dump_equal(a, b):
    da, db = a.dump(), b.dump()
    for k in da:
        np.testing.assert_array_equal(da[k], db[k], err_msg=k)


def test_save_load_resume(torch, tmp_path):
    from paper_2601_11808_gb300.sivf import Index
    w = W.small("sift_window", n_comp=64, nlist=64, slab_size=64)
    ctr = W.centers(w)
    cent = W.index_centroids(w, ctr)
    n, n_max = 8000, 16000
    S = 2 * (n_max // 64 + w.nlist)
    g = Index(w.d, w.nlist, 64, n_max, S, scan_dtypes=("bf16", "fp8"))
    g.set_centroids(torch.from_numpy(cent).cuda())
    x = W.vectors(w, 0, n, ctr)
    ids = W.stream_ids(0, n, n_max)
    g.add(torch.from_numpy(ids).cuda(), torch.from_numpy(x).cuda())
    g.remove(torch.from_numpy(ids[::5]).cuda())
    path = os.path.join(tmp_path, "index.sivf")
    g.save(path)
    h = Index.load(path)
    _dump_equal(g, h)
    _payload_equal(g, h)
    np.testing.assert_array_equal(g.centroids().cpu().numpy(), h.centroids().cpu().numpy())
    q = torch.from_numpy(W.queries(w, 0, 60, ctr)).cuda()
    for form in ("fp32", "bf16", "fp8"):
        da, ia = g.search(q, 10, 6, form)
        db, ib = h.search(q, 10, 6, form)
        np.testing.assert_array_equal(da.cpu().numpy(), db.cpu().numpy())
        np.testing.assert_array_equal(ia.cpu().numpy(), ib.cpu().numpy())
    # resume: the same batches on both, then compare with each other and the oracle
    o = oracle.OracleIVF(w.d, w.nlist, 64, n_max, S)
    o.set_centroids(cent)
    o.add(ids, x)
    o.remove(ids[::5])
    x2 = W.vectors(w, n, 3000, ctr)
    ids2 = W.stream_ids(n, 3000, n_max)
    for idx in (g, h):
        idx.add(torch.from_numpy(ids2).cuda(), torch.from_numpy(x2).cuda())
        idx.remove(torch.from_numpy(ids[1::7]).cuda())
    o.add(ids2, x2)
    o.remove(ids[1::7])
    # physical slab ids depend on the order in which a delete batch pushes
    # emptied slabs (device atomics), so after further batches the two are
    # compared through the logical state the oracle models, and by results
    compare_state(g.dump(), o, 64, S)
    compare_state(h.dump(), o, 64, S)
    da, ia = g.search(q, 10, 6, "fp32")
    db, ib = h.search(q, 10, 6, "fp32")
    np.testing.assert_array_equal(da.cpu().numpy(), db.cpu().numpy())
    np.testing.assert_array_equal(ia.cpu().numpy(), ib.cpu().numpy())
    g.close()
    h.close()


def test_load_refuses_foreign_files(torch, tmp_path):
    from paper_2601_11808_gb300.sivf import Index, SivfError
    with pytest.raises(SivfError):
        Index.load(os.path.join(tmp_path, "missing.sivf"))
    bad = os.path.join(tmp_path, "bad.sivf")
    with open(bad, "wb") as f:
        f.write(b"not a checkpoint" * 8)
    with pytest.raises(SivfError):
        Index.load(bad)
