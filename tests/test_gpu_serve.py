"""GPU tests of the serving loop (sivf_server).

- Same alone and in the mix: a stream of inserts (some carrying evictions of
  the oldest ids), deletes and queries goes through the server, which
  coalesces them into batches and overlaps them on the device.  Each request
  reports the batch that served it.  A twin index then replays the served
  mutation batches in that order, and before each query batch runs every
  query request of it ALONE (its own search call).  The served results must
  equal the alone results (FP32: bit for bit; BF16: within the FP32
  re-rank tolerance, ids equal except at ties), the FP32 ones must match the
  oracle at the same point, and the final index state must equal the
  oracle's bit for bit.
- Admission: with a small slab pool, requests whose batch the device
  rejects get SIVF_E_NOMEM exactly where the oracle, replaying the same
  batches, rejects them.
- Continuous batching: queries submitted together are coalesced.
"""
import numpy as np
import pytest

import oracle
from sivf_check import build_lib, compare_state, compare_topk
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N_MAX = 1 << 17


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def cuda(t, a):
    return t.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(torch, w, S, dtypes):
    from paper_2601_11808_gb300.sivf import Index
    cent = W.index_centroids(w)
    out = []
    for _ in range(2):
        g = Index(w.d, w.nlist, w.slab_size, N_MAX, S, 0, dtypes)
        g.set_centroids(cuda(torch, cent))
        out.append(g)
    o = oracle.OracleIVF(w.d, w.nlist, w.slab_size, N_MAX, S, S)
    o.set_centroids(cent)
    return out[0], out[1], o


def _stream(w, rng, n_req, window, start, qstart):
    """Requests (kind, payload): inserts of fresh ids that evict the oldest
    beyond `window`, deletes of random live ids, queries."""
    ctr = W.centers(w)
    live = list(range(start))           # oldest first
    pos, qpos = start, qstart
    reqs = []
    for _ in range(n_req):
        u = rng.random()
        if u < 0.5:
            n = int(rng.integers(1, 400))
            ids = W.stream_ids(pos, n, N_MAX)
            x = W.vectors(w, pos, n, ctr)
            pos += n
            live += ids.tolist()
            over = max(0, len(live) - window)
            evict = np.asarray(live[:over], np.int64)
            live = live[over:]
            reqs.append(("add", ids, x, evict))
        elif u < 0.65:
            n = int(rng.integers(1, 200))
            pick = rng.choice(len(live), size=min(n, len(live)), replace=False)
            ids = np.asarray([live[i] for i in pick], np.int64)
            gone = set(ids.tolist())
            live = [v for v in live if v not in gone]
            reqs.append(("remove", ids))
        else:
            n = int(rng.integers(1, 60))
            reqs.append(("search", W.queries(w, qpos, n, ctr)))
            qpos += n
    return reqs


def _serve(sv, reqs):
    ids = []
    for r in reqs:
        if r[0] == "add":
            ids.append(sv.add(r[1], r[2], evict=r[3]))
        elif r[0] == "remove":
            ids.append(sv.remove(r[1]))
        else:
            ids.append(sv.search(r[1]))
    return [sv.wait(i) for i in ids]


def _replay(torch, twin, o, reqs, infos, k, P, dtype):
    """Apply the served batches in order on the twin and the oracle; run
    every query request alone at its batch's point."""
    by_batch = {}
    for i, inf in enumerate(infos):
        by_batch.setdefault(inf["batch"], []).append(i)
    for b in sorted(by_batch):
        members = by_batch[b]
        kind = reqs[members[0]][0]
        assert all(reqs[i][0] == kind for i in members)
        if kind == "search":
            for i in members:
                q = reqs[i][1]
                td, ti = twin.search(cuda(torch, q), k, P, dtype)
                td, ti = td.cpu().numpy(), ti.cpu().numpy()
                sd, si = infos[i]["dist"], infos[i]["labels"]
                if dtype == "fp32":
                    np.testing.assert_array_equal(si, ti, err_msg=f"request {i}")
                    np.testing.assert_array_equal(sd, td, err_msg=f"request {i}")
                    od, oi = o.search(q, k, P)
                    compare_topk(sd, si, od, oi, 1e-5, f"request {i}")
                else:
                    compare_topk(sd, si, td.astype(np.float64), ti, 1e-5, f"request {i}")
            continue
        if kind == "add":
            ev = [reqs[i][3] for i in members if len(reqs[i][3])]
            st = 0
            if ev:
                ev = np.concatenate(ev)
                twin.remove(cuda(torch, ev))
                o.remove(ev)
            ids = np.concatenate([reqs[i][1] for i in members])
            x = np.concatenate([reqs[i][2] for i in members])
            try:
                o.add(ids, x)
            except oracle.OracleError as e:
                st = e.status
            from paper_2601_11808_gb300.sivf import SivfError
            try:
                twin.add(cuda(torch, ids), cuda(torch, x), sync=True)
                tst = 0
            except SivfError as e:
                tst = e.status
            assert tst == st
        else:
            ids = np.concatenate([reqs[i][1] for i in members])
            twin.remove(cuda(torch, ids))
            o.remove(ids)
            st = 0
        for i in members:
            assert infos[i]["status"] == st, (i, infos[i], st)


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_results_same_alone_and_in_mix(torch, dtype):
    from paper_2601_11808_gb300.sivf import Server
    w = W.small("tiny_window")
    S = 3000
    g, twin, o = _pair(torch, w, S, ("bf16",))
    n0 = 8000
    ids0, x0 = W.stream_ids(0, n0, N_MAX), W.vectors(w, 0, n0)
    for idx in (g, twin):
        idx.add(cuda(torch, ids0), cuda(torch, x0))
    o.add(ids0, x0)
    g.sync()
    k, P = 10, 6
    reqs = _stream(w, np.random.default_rng(5), 160, n0, n0, 0)
    sv = Server(g, k=k, nprobe=P, dtype=dtype, depth=3, max_query_batch=128,
                max_insert_batch=1024, max_delete_batch=1024)
    infos = _serve(sv, reqs)
    stats = sv.stats()
    sv.close()
    assert all(inf["status"] == 0 for inf in infos)
    assert sum(stats["requests"]) == len(reqs)
    assert sum(stats["batches"]) == len({inf["batch"] for inf in infos})
    for inf in infos:
        assert inf["latency_ms"] >= inf["queue_ms"] >= 0.0
    _replay(torch, twin, o, reqs, infos, k, P, dtype)
    g.sync()
    twin.sync()
    compare_state(g.dump(), o, w.slab_size, S)
    compare_state(twin.dump(), o, w.slab_size, S)


def test_admission_by_free_slabs(torch):
    from paper_2601_11808_gb300.sivf import Server
    w = W.small("tiny_window", nlist=4, n_comp=4)
    S = 40
    g, twin, o = _pair(torch, w, S, ())
    ctr = W.centers(w)
    reqs, pos = [], 0
    rng = np.random.default_rng(1)
    live = []
    for r in range(30):
        if r % 3 == 2 and live:
            n = min(len(live), 300)
            ids = np.asarray(live[:n], np.int64)
            live = live[n:]
            reqs.append(("remove", ids))
        else:
            n = int(rng.integers(100, 600))
            ids = W.stream_ids(pos, n, N_MAX)
            reqs.append(("add", ids, W.vectors(w, pos, n, ctr), np.zeros(0, np.int64)))
            live += ids.tolist()
            pos += n
    sv = Server(g, k=5, nprobe=2, depth=2, max_query_batch=16, max_insert_batch=2048,
                max_delete_batch=2048)
    infos = _serve(sv, reqs)
    stats = sv.stats()
    sv.close()
    # the pool (40 slabs of 32) cannot hold every insert: some are rejected
    assert any(inf["status"] == 2 for inf in infos)
    assert stats["rejected"] == sum(inf["status"] != 0 for inf in infos)
    _replay(torch, twin, o, reqs, infos, 5, 2, "fp32")
    g.sync()
    compare_state(g.dump(), o, w.slab_size, S)


def test_queries_are_coalesced(torch):
    from paper_2601_11808_gb300.sivf import Server
    w = W.small("tiny_window")
    g, twin, o = _pair(torch, w, 2000, ())
    ids0, x0 = W.stream_ids(0, 20000, N_MAX), W.vectors(w, 0, 20000)
    g.add(cuda(torch, ids0), cuda(torch, x0))
    g.sync()
    sv = Server(g, k=10, nprobe=8, depth=2, max_query_batch=256)
    q = W.queries(w, 0, 400)
    reqs = [sv.search(q[i:i + 4]) for i in range(0, 400, 4)]
    infos = [sv.wait(r) for r in reqs]
    st = sv.stats()
    sv.close()
    assert st["requests"][2] == 100
    assert st["batches"][2] < 100          # requests that waited joined one batch
    assert st["items"][2] == 400
    got = np.concatenate([inf["labels"] for inf in infos])
    d, l = g.search(cuda(torch, q), 10, 8)
    np.testing.assert_array_equal(got, l.cpu().numpy())


def test_bad_requests(torch):
    from paper_2601_11808_gb300.sivf import Server, SivfError
    w = W.small("tiny_window")
    g, twin, o = _pair(torch, w, 200, ())
    sv = Server(g, k=4, nprobe=2, depth=1, max_query_batch=8, max_insert_batch=8,
                max_delete_batch=8)
    with pytest.raises(SivfError):
        sv.search(W.queries(w, 0, 9))            # over the query batch limit
    with pytest.raises(SivfError):
        sv.add(np.arange(9), W.vectors(w, 0, 9))
    with pytest.raises(SivfError):
        sv.remove(np.arange(9))
    r = sv.search(W.queries(w, 0, 3))
    inf = sv.wait(r)
    assert inf["status"] == 0 and (inf["labels"] == -1).all()   # empty index
    sv.close()
    with pytest.raises(SivfError):
        Server(g, k=4, nprobe=w.nlist + 1)


def test_idle_compaction(torch):
    """A fragmented index (60 % of its ids deleted at random) handed to a
    server with background compaction: while idle the worker runs passes of
    at most max_insert_batch members until one moves nothing.  The passes
    free and move exactly what the oracle's passes with the same budget do,
    the final state equals the oracle's bit for bit, and searches served
    afterwards equal the oracle's."""
    import time
    from paper_2601_11808_gb300.sivf import Server
    w = W.small("tiny_window")
    S = 2 * (20000 // w.slab_size + w.nlist)
    g, _, o = _pair(torch, w, S, ())
    ids0, x0 = W.stream_ids(0, 20000, N_MAX), W.vectors(w, 0, 20000)
    g.add(cuda(torch, ids0), cuda(torch, x0))
    o.add(ids0, x0)
    gone = W.sample_ids(w.seed, 15, 0, ids0, 12000)
    g.remove(cuda(torch, gone))
    o.remove(gone)
    g.sync()
    budget = 1024
    sv = Server(g, k=10, nprobe=8, depth=2, max_query_batch=256, max_insert_batch=budget,
                compact_min_free=1)
    last, t0 = -1, time.time()
    while time.time() - t0 < 10:
        st = sv.stats()
        if st["compact_passes"] == last and last > 0:
            break
        last = st["compact_passes"]
        time.sleep(0.2)
    q = W.queries(w, 0, 64)
    info = sv.wait(sv.search(q))
    st = sv.stats()
    sv.close()
    freed = moved = passes = 0
    while True:
        fr, mv = o.compact(1, budget)
        if mv == 0:
            break
        freed, moved, passes = freed + fr, moved + mv, passes + 1
    assert passes > 1
    assert (st["compact_passes"], st["compact_freed"], st["compact_moved"]) == (passes, freed, moved)
    g.sync()
    compare_state(g.dump(), o, w.slab_size, S)
    od, oi = o.search(q, 10, 8)
    compare_topk(info["dist"], info["labels"], od, oi, 1e-5, "served after compaction")
