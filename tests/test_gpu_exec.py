"""GPU tests of the mixed-batch executor and of the scan-tile table.

- A queue of uneven add / remove / search batches (each search with its own
  nprobe and dtype) recorded into one CUDA graph leaves the index in the
  state the oracle reaches by applying the same batches in order (bit-exact
  state).  Per-batch statuses and counts equal the oracle's.  FP32 search
  results are within the FP32 tolerance of the oracle's; every search equals
  the same batch run as a single call on a twin index.
- Relaunching after refilling the bound buffers in place runs the new data.
- A batch the slab pool cannot hold is rejected inside the graph with
  SIVF_E_NOMEM and changes nothing; later batches still run.
- Every valid scan tile gives the same search results; the autotuner
  installs a tile that the table then reports.
"""
import numpy as np
import pytest

import oracle
from sivf_check import build_lib, compare_state, compare_topk
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


def cuda(t, a):
    return t.from_numpy(np.ascontiguousarray(a)).cuda()


WT = W.small("tiny_window")
N_MAX = 1 << 16


def _index(torch, w, n_slabs, dtypes=("bf16",)):
    from paper_2601_11808_gb300.sivf import Index
    cent = W.index_centroids(w)
    g = Index(w.d, w.nlist, w.slab_size, N_MAX, n_slabs, 0, dtypes)
    g.set_centroids(cuda(torch, cent))
    return g, cent


def _oracle(w, n_slabs, cent):
    o = oracle.OracleIVF(w.d, w.nlist, w.slab_size, N_MAX, n_slabs, n_slabs)
    o.set_centroids(cent)
    return o


class Stream:
    """Host bookkeeping of a sliding window: fresh ids, the live set."""

    def __init__(self, w, ctr):
        self.w, self.ctr = w, ctr
        self.pos = 0
        self.qpos = 0
        self.live = []
        self.rnd = 0

    def take_add(self, n, overwrite=0):
        ids = W.stream_ids(self.pos, n, N_MAX)
        x = W.vectors(self.w, self.pos, n, self.ctr)
        self.pos += n
        if overwrite and self.live:
            # a few live ids re-added with new vectors: delete-then-insert
            k = min(overwrite, len(self.live), n)
            ids[:k] = np.asarray(self.live[:k], np.int64)
        return ids, x

    def take_remove(self, n):
        self.rnd += 1
        pool = np.asarray(sorted(set(self.live)), np.int64)
        got = W.sample_ids(0, 9, self.rnd, pool, n) if len(pool) else np.zeros(0, np.int64)
        # ids never inserted are no-ops
        extra = np.asarray([N_MAX - 1 - self.rnd], np.int64)
        return np.concatenate([got, extra])[:max(n, 1)]

    def take_queries(self, n):
        q = W.queries(self.w, self.qpos, n, self.ctr)
        self.qpos += n
        return q


def _apply_oracle(o, kind, data):
    try:
        if kind == "add":
            c = o.add(*data)
        else:
            c = o.remove(data[0])
        st = 0
    except oracle.OracleError as e:
        c, st = 0, e.status
    return st, c


def _build_queue(torch, st, sched, dtypes):
    """Device buffers of a queue plus the host copies of its data."""
    ops, host = [], []
    for i, (kind, n, P) in enumerate(sched):
        if kind == "add":
            ids, x = st.take_add(n, overwrite=3 if i % 2 else 0)
            ops.append({"kind": "add", "ids": cuda(torch, ids), "x": cuda(torch, x)})
            host.append(("add", (ids, x)))
            # the host view of the live set follows the queue order
            new = set(ids.tolist())
            st.live = [v for v in st.live if v not in new] + ids.tolist()
        elif kind == "remove":
            ids = st.take_remove(n)
            ops.append({"kind": "remove", "ids": cuda(torch, ids)})
            host.append(("remove", (ids,)))
            gone = set(ids.tolist())
            st.live = [v for v in st.live if v not in gone]
        else:
            q = st.take_queries(n)
            k = 10
            dt = dtypes[i % len(dtypes)]
            ops.append({"kind": "search", "q": cuda(torch, q), "k": k, "nprobe": P,
                        "dtype": dt,
                        "dist": torch.empty((n, k), dtype=torch.float32, device="cuda"),
                        "labels": torch.empty((n, k), dtype=torch.int64, device="cuda")})
            host.append(("search", (q, k, P, dt)))
    return ops, host


def _refill(torch, ops, host, st):
    """New data into the same device buffers (same sizes)."""
    new_host = []
    for i, (op, (kind, data)) in enumerate(zip(ops, host)):
        if kind == "add":
            ids, x = st.take_add(len(data[0]), overwrite=3 if i % 2 else 0)
            op["ids"].copy_(cuda(torch, ids))
            op["x"].copy_(cuda(torch, x))
            new = set(ids.tolist())
            st.live = [v for v in st.live if v not in new] + ids.tolist()
            new_host.append(("add", (ids, x)))
        elif kind == "remove":
            ids = st.take_remove(len(data[0]))
            if len(ids) < len(data[0]):   # pad with absent ids (no-ops)
                ids = np.concatenate([ids, N_MAX - 100 - np.arange(len(data[0]) - len(ids))])
            op["ids"].copy_(cuda(torch, ids))
            gone = set(ids.tolist())
            st.live = [v for v in st.live if v not in gone]
            new_host.append(("remove", (ids,)))
        else:
            q = st.take_queries(len(data[0]))
            op["q"].copy_(cuda(torch, q))
            new_host.append(("search", (q,) + data[1:]))
    return new_host


def _run_and_check(torch, g, twin, o, ex, ops, host):
    ex.launch()
    res = ex.results()
    for i, (op, (kind, data), r) in enumerate(zip(ops, host, res)):
        if kind == "search":
            q, k, P, dt = data
            assert r[0] == 0 and r[1] == len(q)
            gd, gi = op["dist"].cpu().numpy(), op["labels"].cpu().numpy()
            td, ti = twin.search(cuda(torch, q), k, P, dt)
            np.testing.assert_array_equal(gi, ti.cpu().numpy(), err_msg=f"batch {i}")
            np.testing.assert_array_equal(gd, td.cpu().numpy(), err_msg=f"batch {i}")
            if dt == "fp32":
                od, oi = o.search(q, k, P)
                compare_topk(gd, gi, od, oi, 1e-5, f"batch {i}")
        else:
            ost, oc = _apply_oracle(o, kind, data)
            assert (r[0], r[1]) == (ost, oc), f"batch {i} {kind}: {r} vs oracle {ost, oc}"
            if kind == "add":
                twin.add(cuda(torch, data[0]), cuda(torch, data[1]))
            else:
                twin.remove(cuda(torch, data[0]))
        assert r[2] >= 0.0
    twin.sync()
    compare_state(g.dump(), o, g.slab_size, g.n_slabs)
    compare_state(twin.dump(), o, g.slab_size, g.n_slabs)


def test_mixed_queue_matches_oracle_and_single_calls(torch):
    w = WT
    S = 2000
    g, cent = _index(torch, w, S)
    twin, _ = _index(torch, w, S)
    o = _oracle(w, S, cent)
    st = Stream(w, W.centers(w))
    ids, x = st.take_add(6000)
    st.live = ids.tolist()
    for idx in (g, twin):
        idx.add(cuda(torch, ids), cuda(torch, x))
    o.add(ids, x)
    sched = W.mixed_schedule(n_batches=6, max_query=300, max_delete=1500,
                             max_insert=1500, nprobes=(1, 4, 8, 64), seed=3)
    ops, host = _build_queue(torch, st, sched, ("fp32", "bf16"))
    ex = g.executor(ops)
    assert ex.kernels > len(ops)
    _run_and_check(torch, g, twin, o, ex, ops, host)
    # refill the bound buffers in place and replay the same graph
    host2 = _refill(torch, ops, host, st)
    _run_and_check(torch, g, twin, o, ex, ops, host2)
    ex.close()


def test_queue_rejects_oversized_add_and_continues(torch):
    w = W.small("tiny_window", nlist=4, n_comp=4)
    S = 12
    g, cent = _index(torch, w, S, dtypes=())
    o = _oracle(w, S, cent)
    st = Stream(w, W.centers(w))
    a1, x1 = st.take_add(100)
    a2, x2 = st.take_add(1000)          # more slabs than the pool holds
    r1 = a1[:10]
    q = st.take_queries(7)
    ops = [{"kind": "add", "ids": cuda(torch, a1), "x": cuda(torch, x1)},
           {"kind": "add", "ids": cuda(torch, a2), "x": cuda(torch, x2)},
           {"kind": "remove", "ids": cuda(torch, r1)},
           {"kind": "search", "q": cuda(torch, q), "k": 5, "nprobe": 2, "dtype": "fp32",
            "dist": torch.empty((7, 5), dtype=torch.float32, device="cuda"),
            "labels": torch.empty((7, 5), dtype=torch.int64, device="cuda")}]
    ex = g.executor(ops)
    ex.launch()
    res = ex.results()
    exp = [_apply_oracle(o, "add", (a1, x1)), _apply_oracle(o, "add", (a2, x2)),
           _apply_oracle(o, "remove", (r1,))]
    assert exp[1][0] == 2  # the oracle rejects it too (SIVF_E_NOMEM)
    assert [(r[0], r[1]) for r in res[:3]] == exp
    assert res[3][:2] == (0, 7)
    compare_state(g.dump(), o, w.slab_size, S)
    od, oi = o.search(q, 5, 2)
    compare_topk(ops[3]["dist"].cpu().numpy(), ops[3]["labels"].cpu().numpy(), od, oi, 1e-5)
    ex.close()


def test_queue_argument_errors(torch):
    from paper_2601_11808_gb300.sivf import SivfError
    g, cent = _index(torch, WT, 100)
    q = cuda(torch, W.queries(WT, 0, 3))
    bad = [{"kind": "search", "q": q, "k": 5, "nprobe": WT.nlist + 1, "dtype": "fp32",
            "dist": torch.empty((3, 5), dtype=torch.float32, device="cuda"),
            "labels": torch.empty((3, 5), dtype=torch.int64, device="cuda")}]
    with pytest.raises(SivfError):
        g.executor(bad)
    with pytest.raises(SivfError):     # 4k > 512: no reduced-precision scan for k = 200
        g.executor([dict(bad[0], nprobe=2, k=200, dtype="bf16",
                         dist=torch.empty((3, 200), dtype=torch.float32, device="cuda"),
                         labels=torch.empty((3, 200), dtype=torch.int64, device="cuda"))])


def _t(tq, spc, ips, sel, nf=0):
    return dict(queries_per_tile=tq, slabs_per_chunk=spc, items_per_sm=ips,
                select_slabs=sel, nearest_first=nf)


# (d = 128, slab 64, k = 10): all fit in shared memory
FP32_TILES = [_t(8, 1, 1, 1), _t(16, 2, 16, 4), _t(8, 8, 4, 8), _t(32, 16, 2, 2),
              _t(64, 4, 8, 1)]
# vector-row scan one launch / nearest list first / seeded; query-row scan
TC_TILES = [_t(64, 1, 16, 0, 0), _t(64, 8, 1, 0, 1), _t(64, 4, 4, 0, 2), _t(128, 4, 4, 0, 1),
            _t(128, 2, 8, 2, 0)]


@pytest.fixture(scope="module")
def filled(torch):
    w = W.small("sift_window", n_comp=64, nlist=64, slab_size=64)
    S = 400
    from paper_2601_11808_gb300.sivf import Index
    cent = W.index_centroids(w)
    g = Index(w.d, w.nlist, w.slab_size, N_MAX, S, 0, ("bf16",))
    g.set_centroids(cuda(torch, cent))
    o = oracle.OracleIVF(w.d, w.nlist, w.slab_size, N_MAX, S)
    o.set_centroids(cent)
    x = W.vectors(w, 0, 9000)
    ids = W.stream_ids(0, 9000, N_MAX)
    g.add(cuda(torch, ids), cuda(torch, x))
    o.add(ids, x)
    g.remove(cuda(torch, ids[::4]))
    o.remove(ids[::4])
    g.sync()
    return w, g, o


@pytest.mark.parametrize("ti", range(len(FP32_TILES)))
@pytest.mark.parametrize("nq,P", [(5, 3), (300, 8), (2000, 20)])
def test_fp32_tiles_give_oracle_results(torch, filled, ti, nq, P):
    w, g, o = filled
    q = W.queries(w, 0, nq)
    g.set_tile("fp32", nq, 10, P, FP32_TILES[ti])
    assert g.get_tile("fp32", nq, 10, P) == FP32_TILES[ti]
    gd, gi = g.search(cuda(torch, q), 10, P)
    g.set_tile("fp32", nq, 10, P, None)
    od, oi = o.search(q, 10, P)
    compare_topk(gd.cpu().numpy(), gi.cpu().numpy(), od, oi, 1e-5, f"tile {ti}")


@pytest.mark.parametrize("ti", range(len(TC_TILES)))
@pytest.mark.parametrize("nq,P", [(5, 3), (1000, 8)])
def test_tc_tiles_do_not_change_results(torch, filled, ti, nq, P):
    w, g, o = filled
    q = cuda(torch, W.queries(w, 0, nq))
    ref_d, ref_i = g.search(q, 10, P, "bf16")
    g.set_tile("bf16", nq, 10, P, TC_TILES[ti])
    gd, gi = g.search(q, 10, P, "bf16")
    g.set_tile("bf16", nq, 10, P, None)
    np.testing.assert_array_equal(gi.cpu().numpy(), ref_i.cpu().numpy())
    np.testing.assert_array_equal(gd.cpu().numpy(), ref_d.cpu().numpy())


def test_bad_tiles_rejected(torch, filled):
    from paper_2601_11808_gb300.sivf import SivfError
    w, g, o = filled
    for t in [_t(12, 1, 1, 1), _t(8, 0, 1, 1), _t(8, 1, 17, 1), _t(8, 1, 1, 9),
              _t(32, 1, 1, 4)]:          # the last needs 274 KB of shared memory
        with pytest.raises(SivfError):
            g.set_tile("fp32", 100, 10, 8, t)
    for t in [_t(64, 1, 1, 0, 3), _t(48, 1, 1, 0, 1), _t(128, 1, 1, 4, 1)]:
        with pytest.raises(SivfError):
            g.set_tile("bf16", 100, 10, 8, t)


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_autotune_installs_a_tile(torch, filled, dtype):
    w, g, o = filled
    nq, P = 500, 8
    q = W.queries(w, 100, nq)
    tile, ms = g.autotune(cuda(torch, q), 10, P, dtype, reps=2)
    assert ms > 0
    assert g.get_tile(dtype, nq, 10, P) == tile
    gd, gi = g.search(cuda(torch, q), 10, P, dtype)
    if dtype == "fp32":
        od, oi = o.search(q, 10, P)
        compare_topk(gd.cpu().numpy(), gi.cpu().numpy(), od, oi, 1e-5)
    g.set_tile(dtype, nq, 10, P, None)


def test_bucket_rule_matches_library(torch, filled):
    """autotune.bucket names the library's table slots: shapes in one bucket
    share a tile, shapes in another do not."""
    from paper_2601_11808_gb300 import autotune
    w, g, o = filled
    t = _t(16, 4, 2, 1)
    shapes = [(40, 8), (50, 8), (63, 8), (64, 8), (20, 16), (40, 16), (1, 8), (2, 1)]
    g.set_tile("fp32", 40, 10, 8, t)
    b0 = autotune.bucket(w.nlist, 40, 10, 8, "fp32")
    for nq, P in shapes:
        same = autotune.bucket(w.nlist, nq, 10, P, "fp32") == b0
        assert (g.get_tile("fp32", nq, 10, P) == t) == same, (nq, P)
    # the kept-candidate bucket: k = 10 and k = 17 differ for fp32 (<= 16 / <= 64)
    assert g.get_tile("fp32", 40, 17, 8) != t
    g.set_tile("fp32", 40, 10, 8, None)


def test_tune_cache_round_trip(torch, filled, tmp_path):
    from paper_2601_11808_gb300 import autotune
    w, g, o = filled
    q = cuda(torch, W.queries(w, 0, 256))
    path = str(tmp_path / "tiles.json")
    shapes = [(256, 10, 8, "fp32"), (160, 10, 16, "fp32"), (16, 10, 4, "bf16")]
    got = autotune.tune(g, q, shapes, cache_path=path, reps=1)
    assert len(got) == 2          # the first two shapes share a bucket
    for nq, k, P, dt in shapes:
        g.set_tile(dt, nq, k, P, None)
    again = autotune.tune(g, q, shapes, cache_path=path, reps=1)
    assert again == got           # read back, not re-timed
    for nq, k, P, dt in shapes:
        assert g.get_tile(dt, nq, k, P) == got[autotune.bucket(w.nlist, nq, k, P, dt)]["tile"]
    for nq, k, P, dt in shapes:
        g.set_tile(dt, nq, k, P, None)


def test_queue_with_compaction_passes(torch):
    """Compaction passes recorded in a queue between its batches: each pass
    moves what the oracle's pass moves at the same point (the result's
    count), searches after it match the oracle, and the final state is
    bit-exact."""
    w = WT
    S = 1500
    g, cent = _index(torch, w, S)
    o = _oracle(w, S, cent)
    st = Stream(w, W.centers(w))
    ids, x = st.take_add(12000)
    g.add(cuda(torch, ids), cuda(torch, x))
    o.add(ids, x)
    rng = np.random.default_rng(5)
    r1 = rng.choice(ids, 7000, replace=False)
    a2, x2 = st.take_add(2000)
    r2 = rng.choice(np.setdiff1d(ids, r1), 1500, replace=False)
    q = st.take_queries(50)
    dist = torch.empty((50, 10), dtype=torch.float32, device="cuda")
    lab = torch.empty((50, 10), dtype=torch.int64, device="cuda")
    ops = [{"kind": "remove", "ids": cuda(torch, r1)},
           {"kind": "compact", "min_free": 1, "max_moves": 1500},
           {"kind": "compact", "min_free": 2, "max_moves": 1 << 20},
           {"kind": "search", "q": cuda(torch, q), "k": 10, "nprobe": 8, "dtype": "fp32",
            "dist": dist, "labels": lab},
           {"kind": "add", "ids": cuda(torch, a2), "x": cuda(torch, x2)},
           {"kind": "remove", "ids": cuda(torch, r2)},
           {"kind": "compact", "min_free": 1, "max_moves": 1 << 20}]
    ex = g.executor(ops)
    ex.launch()
    res = ex.results()
    ex.close()
    exp = [(0, o.remove(r1))]
    exp.append((0, o.compact(1, 1500)[1]))
    exp.append((0, o.compact(2, 1 << 20)[1]))
    od, oi = o.search(q, 10, 8)
    exp.append((0, 50))
    exp.append((0, o.add(a2, x2)))
    exp.append((0, o.remove(r2)))
    exp.append((0, o.compact(1, 1 << 20)[1]))
    assert [(r[0], r[1]) for r in res] == exp
    assert exp[1][1] > 0 and exp[6][1] > 0
    compare_topk(dist.cpu().numpy(), lab.cpu().numpy(), od, oi, 1e-5, "search after passes")
    g.sync()
    compare_state(g.dump(), o, w.slab_size, S)
