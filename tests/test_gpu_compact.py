"""GPU parity of compaction of partly-live slabs against the oracle.

After random deletes, a compaction pass (min_free, max_moves) must select
the same lists, free the same number of slabs and rewrite the same members
as the oracle, and leave the device state equal to the oracle's bit for bit
(members in order, slab positions, dense slots, fill/live, free slabs); the
moved rows keep their FP32 payload and their BF16 / FP8 codes (the codes of
a list do not change when its members move inside it); every search form
returns what it returned before the pass; inserts after it fill the open
last slab.
"""
import numpy as np
import pytest

import oracle
from sivf_check import Pair, build_lib, compare_topk, cuda
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def _filled(torch, w, n, frac, seed):
    ctr = W.centers(w)
    cent = W.index_centroids(w, ctr)
    n_max = 2 * n
    S = 2 * (n // w.slab_size + w.nlist)
    p = Pair(torch, w.d, w.nlist, w.slab_size, n_max, S, cent, dtypes=("bf16", "fp8"))
    X = W.vectors(w, 0, n + 3000, ctr)
    for b in range(0, n, 10_000):
        p.add(W.stream_ids(b, min(10_000, n - b), n_max), X[b:b + 10_000][: n - b])
    gone = W.sample_ids(w.seed, 14, seed, W.stream_ids(0, n, n_max), int(frac * n))
    p.remove(gone)
    p.check()
    return p, X, ctr, cent


def _payload_rows(p, X, cent):
    """Device payload rows of every live id equal the vector and the oracle's
    encoders of it."""
    pay = p.g.dump_payload(bf16=True, fp8=True)
    dump = p.g.dump()
    att = dump["att"]
    live = np.nonzero(att >= 0)[0]
    rows = (att[live] >> 32) * p.C + (att[live] & 0xffffffff)
    np.testing.assert_array_equal(pay["x32"][rows], X[live])
    np.testing.assert_array_equal(pay["xb16"][rows], oracle.to_bf16(X[live]))
    lists = dump["slab_meta"][att[live] >> 32, 0]
    inv = pay["inv_scale"]
    for l in np.unique(lists)[:12]:
        sel = lists == l
        resid = (X[live[sel]] - cent[l]).astype(np.float32)
        np.testing.assert_array_equal(pay["x8"][rows[sel]], oracle.to_e4m3(resid, inv[l]))


@pytest.mark.parametrize("frac", [0.3, 0.7])
def test_compact_state_payload_and_search(torch, frac):
    w = W.CONFIGS["tiny_window"]
    p, X, ctr, cent = _filled(torch, w, 20_000, frac, int(frac * 10))
    q = W.queries(w, 0, 150, ctr)
    before = {form: p.g.search(cuda(torch, q), 10, 6, form) for form in ("fp32", "bf16", "fp8")}
    before = {f: (d.cpu().numpy(), i.cpu().numpy()) for f, (d, i) in before.items()}
    freed, moved = p.compact(min_free=1)
    assert freed > 0 and moved > 0
    p.check()
    _payload_rows(p, X, cent)
    # nothing left to free
    assert p.compact(min_free=1) == (0, 0)
    # the same results in every form: FP32 bit for bit; the reduced forms
    # keep the same candidates up to ties (slot order changed), and their
    # re-ranked distances are exact FP32
    for form, (bd, bi) in before.items():
        gd, gi = p.g.search(cuda(torch, q), 10, 6, form)
        gd, gi = gd.cpu().numpy(), gi.cpu().numpy()
        if form == "fp32":
            np.testing.assert_array_equal(gd, bd)
            np.testing.assert_array_equal(gi, bi)
        else:
            np.testing.assert_allclose(gd, bd, rtol=1e-6, atol=0)
    compare_topk(*p.search(q, 10, 6), RTOL, "after compaction")
    # inserts continue in the open last slab of each list, as the oracle says
    n = 20_000
    p.add(W.stream_ids(n, 3000, 2 * n), X[n:n + 3000])
    p.check()
    p.remove(W.stream_ids(n, 1000, 2 * n))
    p.check()
    compare_topk(*p.search(q, 10, 6), RTOL, "after more batches")


def test_compact_budget_and_threshold_match_oracle(torch):
    w = W.CONFIGS["tiny_window"]
    p, X, ctr, cent = _filled(torch, w, 20_000, 0.6, 3)
    sizes = [p.o.list_size(l) for l in range(w.nlist)]
    # a budget below the first candidate list's size compacts nothing
    assert p.compact(min_free=1, max_moves=1) == (0, 0)
    p.check()
    # a budget that stops inside the list sequence, then a high threshold
    p.compact(min_free=1, max_moves=int(2.5 * np.mean(sizes)))
    p.check()
    p.compact(min_free=8)
    p.check()
    p.compact(min_free=2, max_moves=4000)
    p.check()
    p.compact(min_free=1)
    p.check()
    compare_topk(*p.search(W.queries(w, 0, 60, ctr), 10, 64), RTOL, "exact after passes")


def test_compact_long_lists_zipf(torch):
    """Skewed lists past 256 slabs (the slab-base scan of one list spans
    several blocks of 256 slabs) and a slab size of 64."""
    w = W.small("tiny_window", d=48, n_comp=16, nlist=16, slab_size=64, zipf=1.3)
    p, X, ctr, cent = _filled(torch, w, 60_000, 0.5, 5)
    assert max(len(p.o.list_slabs(l)[0]) for l in range(w.nlist)) > 256
    p.compact(min_free=1)
    p.check()
    _payload_rows(p, X, cent)
    compare_topk(*p.search(W.queries(w, 0, 80, ctr), 10, 3), RTOL, "zipf compacted")
