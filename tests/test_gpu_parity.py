"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Index state (assignment, list membership and order, slab positions, slab
fill/live, free slabs) must match bit for bit; search distances within a
relative 1e-5 (FP32 direct-form sums of squares of at most 256 terms carry
a relative error below (d + 1) 2^-24 = 1.5e-5 in the worst case at d = 256
and far less in practice), id sets equal except at distance ties inside
that tolerance.
"""
import numpy as np
import pytest

import oracle
from sivf_check import Pair, build_lib, check_invariants, compare_topk, cuda
from paper_2601_11808_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    build_lib()
    return t


# ------------------------------------------------------------ coarse steps
def _assign_cases():
    rng = np.random.default_rng(0)
    yield "mixture", W.index_centroids(W.small()), W.vectors(W.small(), 0, 5000)
    # small integers: many exact ties, resolved to the lowest index
    yield "int_ties", rng.integers(-2, 3, (40, 4)).astype(np.float32), \
        rng.integers(-2, 3, (3000, 4)).astype(np.float32)
    c = rng.standard_normal((33, 8)).astype(np.float32)
    yield "dup_centroids", np.concatenate([c, c, c]), \
        rng.standard_normal((2000, 8)).astype(np.float32)
    w = W.small("sift_window")
    yield "sift", W.index_centroids(w), W.vectors(w, 0, 4000)
    # points placed exactly half way between two centroids
    a = rng.standard_normal((50, 16)).astype(np.float32)
    b = a + np.float32(2.0)
    mid = ((a + b) / 2).astype(np.float32)
    yield "midpoints", np.concatenate([a, b]), mid
    yield "one_list", rng.standard_normal((1, 12)).astype(np.float32), \
        rng.standard_normal((100, 12)).astype(np.float32)
    # d % 16 == 0 takes the BF16 tensor-core first stage: duplicated
    # centroids and integer grids with many exact ties (more candidates than
    # the warp selection holds take its serial FP64 path)
    c16 = rng.standard_normal((33, 16)).astype(np.float32)
    yield "dup_centroids_d16", np.concatenate([c16] * 5), \
        rng.standard_normal((2000, 16)).astype(np.float32)
    yield "int_ties_d32", rng.integers(-2, 3, (300, 32)).astype(np.float32), \
        rng.integers(-2, 3, (3000, 32)).astype(np.float32)
    # the fused first stage for assignment (64 <= d <= 128): more row tiles
    # of 128 than SMs (each CTA loops over tiles), 300 lists in two chunks
    # of 256 (the second ragged)
    c64 = rng.standard_normal((300, 64)).astype(np.float32)
    yield "many_rows_d64", c64, \
        (c64[rng.integers(0, 300, 25000)]
         + 0.3 * rng.standard_normal((25000, 64))).astype(np.float32)
    # d = 96: the second 64-column TMA box is half outside the rows
    c96 = rng.standard_normal((700, 96)).astype(np.float32)
    yield "d96", c96, (c96[rng.integers(0, 700, 3000)]
                       + 0.5 * rng.standard_normal((3000, 96))).astype(np.float32)
    # 150 copies of one centroid among 400 others (the median spacing keeps
    # the single BF16 stage): the fused stage's per-thread lists overflow,
    # the row is redone from all lists (and its set of more than 128
    # candidates takes the serial FP64 path)
    one = rng.standard_normal((1, 64)).astype(np.float32)
    oth = rng.standard_normal((400, 64)).astype(np.float32)
    yield "identical_150_d64", np.concatenate([oth[:200], np.repeat(one, 150, 0), oth[200:]]), \
        (one + 0.05 * rng.standard_normal((500, 64))).astype(np.float32)
    # integer grid: exact ties between lists, several candidates per row
    yield "int_ties_d64", rng.integers(-1, 2, (400, 64)).astype(np.float32), \
        rng.integers(-1, 2, (3000, 64)).astype(np.float32)
    # 2,048 lists around 64 mixture centers (sigma 0.1, d = 128): the single
    # BF16 bound is wider than the centroid spacing, so assignment takes the
    # split first stage
    w = W.small("mixed_batches")
    yield "clustered_d128", W.index_centroids(w), W.vectors(w, 0, 3000)


# first stage of assignment (sivf_assign_stage) the centroids above select:
# 1 single BF16, 3 split BF16
STAGE = {"sift": 1, "int_ties_d32": 1, "many_rows_d64": 1, "d96": 1, "identical_150_d64": 1,
         "int_ties_d64": 1, "clustered_d128": 3}


@pytest.mark.parametrize("case", [c[0] for c in _assign_cases()])
def test_assign_bit_exact(torch, case):
    cent, x = {c[0]: c[1:] for c in _assign_cases()}[case]
    from paper_2601_11808_gb300.sivf import Index
    g = Index(cent.shape[1], cent.shape[0], 32, 100, 10)
    g.set_centroids(cuda(torch, cent))
    o = oracle.OracleIVF(cent.shape[1], cent.shape[0], n_max=10, n_slabs=10)
    o.set_centroids(cent)
    got = g.assign(cuda(torch, x)).cpu().numpy()
    np.testing.assert_array_equal(got, o.assign(x))
    if case in STAGE:
        from paper_2601_11808_gb300.sivf import sivf_assign_stage
        assert sivf_assign_stage(g.h) == STAGE[case]


@pytest.mark.parametrize("P", [1, 5, 8])
def test_probe_sets_bit_exact_d16(torch, P):
    """d = 16 with heavy ties: P = 1 takes the BF16 tensor-core first stage
    (FP32 recheck, FP64 near-ties), P > 1 the FP32 first stage."""
    rng = np.random.default_rng(100 + P)
    cent = rng.integers(-3, 4, (300, 16)).astype(np.float32)   # heavy ties
    q = rng.integers(-3, 4, (700, 16)).astype(np.float32)
    from paper_2601_11808_gb300.sivf import Index
    g = Index(16, 300, 32, 100, 10)
    g.set_centroids(cuda(torch, cent))
    o = oracle.OracleIVF(16, 300, n_max=10, n_slabs=10)
    o.set_centroids(cent)
    got = g.probe(cuda(torch, q), P).cpu().numpy()
    np.testing.assert_array_equal(np.sort(got, axis=1), np.sort(o.probe(q, P), axis=1))


@pytest.mark.parametrize("P", [1, 7, 64, 200])
def test_probe_sets_bit_exact(torch, P):
    rng = np.random.default_rng(P)
    cent = rng.integers(-3, 4, (256, 8)).astype(np.float32)   # heavy ties
    q = rng.integers(-3, 4, (500, 8)).astype(np.float32)
    from paper_2601_11808_gb300.sivf import Index
    g = Index(8, 256, 32, 100, 10)
    g.set_centroids(cuda(torch, cent))
    o = oracle.OracleIVF(8, 256, n_max=10, n_slabs=10)
    o.set_centroids(cent)
    got = g.probe(cuda(torch, q), P).cpu().numpy()
    want = np.sort(o.probe(q, P), axis=1)
    np.testing.assert_array_equal(np.sort(got, axis=1), want)
    # listed nearest first: the FP64 distance never decreases along a row
    for r in range(len(q)):
        d = [float(((q[r].astype(np.float64) - cent[c]) ** 2).sum()) for c in got[r]]
        assert all(d[i] <= d[i + 1] + 1e-9 for i in range(len(d) - 1))


# --------------------------------------------------- tiny sliding window
def test_tiny_window_state_and_search(torch):
    """The tiny sliding-window workload in full: 20,000 vectors d=32,
    nlist=64, slab 32; 10 steps of +2,000 / -2,000 oldest; state compared
    after every batch; 200 queries, k=10, nprobe=8."""
    w = W.CONFIGS["tiny_window"]
    ctr = W.centers(w)
    n_max = 2 * w.window
    S = 2 * (w.window // w.slab_size + w.nlist)
    p = Pair(torch, w.d, w.nlist, w.slab_size, n_max, S, W.index_centroids(w, ctr))
    for b in range(0, w.window, 5000):
        p.add(W.stream_ids(b, 5000, n_max), W.vectors(w, b, 5000, ctr))
        p.check()
    for s in range(10):
        new = w.window + s * w.step
        p.add(W.stream_ids(new, w.step, n_max), W.vectors(w, new, w.step, ctr))
        p.check()
        p.remove(W.stream_ids(new - w.window, w.step, n_max))
        p.check()
    q = W.queries(w, 0, w.n_queries, ctr)
    gd, gi, od, oi = p.search(q, w.k, 8)
    compare_topk(gd, gi, od, oi, RTOL, "tiny P=8")
    for P in (1, 3, 64):
        compare_topk(*p.search(q, w.k, P), RTOL, f"tiny P={P}")
    # nprobe = nlist is exact kNN
    gd, gi = p.g.search(cuda(torch, q), 25, w.nlist)
    ed, ei = p.o.exact_knn(q, 25)
    compare_topk(gd.cpu().numpy(), gi.cpu().numpy(), ed, ei, RTOL, "exact")


@pytest.mark.parametrize("C,d,nq", [(32, 32, 3), (64, 128, 700), (128, 96, 50),
                                    (64, 256, 40), (32, 4, 900), (128, 128, 2000)])
def test_scan_tile_shapes_and_ragged_tails(torch, C, d, nq):
    """Slab sizes 32/64/128, dimensions 4..256 and query counts that select
    every query-tile width and leave ragged tiles and slabs."""
    rng = np.random.default_rng(C + d)
    L = 24
    cent = rng.standard_normal((L, d)).astype(np.float32)
    n = 5 * C * L + 17
    x = (cent[rng.integers(0, L, n)] + 0.5 * rng.standard_normal((n, d))).astype(np.float32)
    p = Pair(torch, d, L, C, 2 * n, 4 * (n // C + L), cent)
    p.add(np.arange(n), x)
    p.remove(np.arange(0, n, 3))
    p.check()
    q = (cent[rng.integers(0, L, nq)] + 0.5 * rng.standard_normal((nq, d))).astype(np.float32)
    for k, P in ((1, 1), (10, 4), (37, L)):
        compare_topk(*p.search(q, k, P), RTOL, f"C{C} d{d} k{k} P{P}")


# ------------------------------------------------------------- edge cases
def test_edge_cases(torch):
    from paper_2601_11808_gb300.sivf import Index, SivfError
    rng = np.random.default_rng(5)
    d, L, C = 8, 4, 32
    cent = rng.standard_normal((L, d)).astype(np.float32)
    p = Pair(torch, d, L, C, 1000, 40, cent)
    q = rng.standard_normal((5, d)).astype(np.float32)
    # empty index: everything padded
    gd, gi, od, oi = p.search(q, 7, L)
    assert (gi == -1).all() and np.isinf(gd).all()
    # duplicates inside a batch: the last occurrence wins
    p.add([3, 3, 5, 3], rng.standard_normal((4, d)))
    p.check()
    # overwrite of a live id: delete-then-insert
    p.add([5, 900], rng.standard_normal((2, d)) + 3)
    p.check()
    # k larger than the live count
    compare_topk(*p.search(q, 50, L), RTOL, "k>n")
    # removes: absent, repeated, mixed
    p.remove([3, 3, 77, 5])
    p.remove([3])
    p.check()
    # ids out of range reject the whole batch, nothing changes
    p.add([1, 1000], rng.standard_normal((2, d)))
    p.remove([900, -1])
    p.check()
    # ragged batch sizes around the rank tile of 1024
    base = 0
    for n in (1, 1023, 1024, 1025, 31):
        ids = np.arange(base, base + n) % 1000
        p.add(ids, rng.standard_normal((n, d)))
        p.check()
        base += n
    p.remove(np.arange(0, 1000, 2))
    p.check()
    # pool exhaustion: the whole batch is refused, state unchanged
    st = p.add(np.arange(1000), rng.standard_normal((1000, d)))
    assert st == 2
    p.check()
    # delete everything: every slab back in the pool
    p.remove(np.arange(1000))
    p.check()
    assert p.g.stats()["free_slabs"] == 40
    # bad host arguments never reach the device
    with pytest.raises(SivfError):
        p.g.search(cuda(torch, q), 0, 1)
    with pytest.raises(SivfError):
        p.g.search(cuda(torch, q), 5, L + 1)
    # set_centroids required first
    g2 = Index(d, L, C, 100, 10)
    with pytest.raises(SivfError) as e:
        g2.add(cuda(torch, np.arange(2)), cuda(torch, np.zeros((2, d), np.float32)))
    assert e.value.status == 3


def test_directory_capacity(torch):
    rng = np.random.default_rng(6)
    cent = np.array([[0] * 4, [10] * 4], np.float32)
    p = Pair(torch, 4, 2, 32, 1000, 50, cent, dir_cap=3)
    p.add(np.arange(96), np.zeros((96, 4)))          # three full slabs
    p.check()
    assert p.add([500], np.zeros((1, 4))) == 2       # a fourth would exceed
    p.add([501], np.full((1, 4), 10.0))              # the other list is fine
    p.remove(np.arange(32))                          # oldest slab freed
    p.add([502], np.zeros((1, 4)))
    p.check()


def test_search_with_probes_skips_invalid_and_duplicate_lists(torch):
    rng = np.random.default_rng(8)
    d, L = 16, 10
    cent = rng.standard_normal((L, d)).astype(np.float32)
    x = rng.standard_normal((3000, d)).astype(np.float32)
    p = Pair(torch, d, L, 64, 5000, 200, cent)
    p.add(np.arange(3000), x)
    q = rng.standard_normal((100, d)).astype(np.float32)
    probes = rng.integers(-2, L + 2, (100, 6)).astype(np.int32)
    probes[:, 3] = probes[:, 1]
    gd, gi = p.g.search_with_probes(cuda(torch, q), 12, cuda(torch, probes))
    clean = np.where((probes >= 0) & (probes < L), probes, -1)
    od, oi = p.o.search_with_probes(q, 12, clean)
    compare_topk(gd.cpu().numpy(), gi.cpu().numpy(), od, oi, RTOL, "given probes")


# ------------------------------------------ full-size SIFT-shaped window
@pytest.mark.parametrize("P", [8, 32])
def test_sift_window_full_size_sampled(torch, P):
    """The SIFT-shaped window at full size (1,000,000 vectors d=128,
    nlist=1024, slab 64) after two +10,000 / -10,000 steps, in the launch
    configuration the benchmark times (10,000 queries, k=10).  Sampled
    outputs are recomputed by the oracle one by one: assignments of sampled
    vectors, probe sets of sampled queries, and their exact top-k over the
    members of the probed lists (walking the window in ascending FP64
    distance and asking the oracle for each vector's list)."""
    w = W.CONFIGS["sift_window"]
    ctr = W.centers(w)
    cent = W.index_centroids(w, ctr)
    n_max = w.window + 4 * w.step
    S = int(1.25 * (w.window // w.slab_size + 2 * w.nlist))
    from paper_2601_11808_gb300.sivf import Index
    g = Index(w.d, w.nlist, w.slab_size, n_max, S)
    g.set_centroids(cuda(torch, cent))
    X = W.vectors(w, 0, w.window + 2 * w.step, ctr)
    for b in range(0, w.window, 100_000):
        g.add(cuda(torch, W.stream_ids(b, 100_000, n_max)), cuda(torch, X[b:b + 100_000]))
    for s in range(2):
        new = w.window + s * w.step
        g.add(cuda(torch, W.stream_ids(new, w.step, n_max)), cuda(torch, X[new:new + w.step]))
        g.remove(cuda(torch, W.stream_ids(s * w.step, w.step, n_max)))
    assert g.sync() == w.step
    live = np.arange(2 * w.step, w.window + 2 * w.step)      # stream positions
    o = oracle.OracleIVF(w.d, w.nlist, n_max=10, n_slabs=10)
    o.set_centroids(cent)
    # sampled assignments (the device address table gives each id's slab)
    dump = g.dump()
    rng = np.random.default_rng(1)
    pos = rng.choice(live, 2000, replace=False)
    att = dump["att"][pos % n_max]
    assert (att >= 0).all()
    lists = dump["slab_meta"][att >> 32, 0]
    np.testing.assert_array_equal(lists, o.assign(X[pos]))
    # the benchmark's launch: 10,000 queries
    Q = W.queries(w, 0, w.n_queries, ctr)
    gd, gi = g.search(cuda(torch, Q), w.k, P)
    gd, gi = gd.cpu().numpy(), gi.cpu().numpy()
    probes = g.probe(cuda(torch, Q[:200]), P).cpu().numpy()
    sample = rng.choice(w.n_queries, 25, replace=False)
    np.testing.assert_array_equal(np.sort(probes[:25], axis=1), np.sort(o.probe(Q[:25], P), axis=1))
    Xl = X[live]
    for r in sample:
        pr = set(o.probe(Q[r:r + 1], P)[0].tolist())
        dd = oracle.dists(Q[r], Xl)
        order = np.argsort(dd, kind="stable")
        od, oi = [], []
        for j in order:
            if int(o.assign(Xl[j:j + 1])[0]) in pr:
                od.append(dd[j])
                oi.append(int(live[j] % n_max))
                if len(od) == w.k:
                    break
        compare_topk(gd[r:r + 1], gi[r:r + 1], np.array([od]), np.array([oi]), RTOL,
                     f"sift q{r}")
    check_invariants(dump, w.slab_size, S)
