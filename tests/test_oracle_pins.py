"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against exact rational arithmetic, brute force
written with numpy, a plain set model of the add/remove semantics, torch's
own bfloat16 / float8 casts, or closed forms.  A plausible mistake in the
oracle (a dropped coordinate, a wrong sign, ties to the wrong index, a top-k
off by one, a slab never returned to the pool, ...) fails at least one of
them; ``test_oracle_mutants.py`` plants such mistakes to show it.
"""
from fractions import Fraction

import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
from oracle import OracleIVF, OracleError


# ---------------------------------------------------------------- helpers
def exact_sq(a, b):
    """Exact squared L2 distance of two float32 vectors (rational)."""
    return sum((Fraction(float(x)) - Fraction(float(y))) ** 2
               for x, y in zip(a, b))


def exact_nearest(x, cent):
    ds = [exact_sq(x, c) for c in cent]
    m = min(ds)
    return ds.index(m)          # first index at the minimum


def exact_probes(q, cent, P):
    ds = [(exact_sq(q, c), i) for i, c in enumerate(cent)]
    ds.sort()
    return [i for _, i in ds[:P]]


def brute_knn(q, x, ids, k):
    """k nearest by (float64 distance, id) -- numpy brute force."""
    q64, x64 = q.astype(np.float64), x.astype(np.float64)
    out_d = np.full((len(q), k), np.inf)
    out_i = np.full((len(q), k), -1, np.int64)
    for r in range(len(q)):
        dd = ((x64 - q64[r]) ** 2).sum(axis=1)
        order = np.lexsort((ids, dd))[:k]
        out_d[r, :len(order)] = dd[order]
        out_i[r, :len(order)] = ids[order]
    return out_d, out_i


def grid_points(rng, n, d, lo=-4, hi=4, denom=1):
    return (rng.integers(lo, hi + 1, size=(n, d)) / denom).astype(np.float32)


# ------------------------------------------------------- coarse quantizer
@pytest.mark.parametrize("d,denom", [(1, 1), (2, 1), (3, 2), (4, 8)])
def test_assign_matches_exact_rational_argmin(d, denom):
    """Small integer / dyadic grids: many exact ties, all resolved to the
    lowest centroid index, as the rational argmin does."""
    rng = np.random.default_rng(100 + d)
    cent = grid_points(rng, 9, d, denom=denom)
    x = grid_points(rng, 300, d, denom=denom)
    o = OracleIVF(d, len(cent), n_max=1000)
    o.set_centroids(cent)
    got = o.assign(x)
    want = [exact_nearest(v, cent) for v in x]
    assert list(got) == want
    # ties really occur in this sample
    n_ties = sum(1 for v in x
                 if sorted(exact_sq(v, c) for c in cent)[:2][0]
                 == sorted(exact_sq(v, c) for c in cent)[:2][1])
    assert n_ties > 0


def test_assign_general_floats_exact_rational():
    rng = np.random.default_rng(7)
    cent = rng.standard_normal((16, 4)).astype(np.float32)
    x = rng.standard_normal((200, 4)).astype(np.float32)
    o = OracleIVF(4, 16, n_max=1000)
    o.set_centroids(cent)
    assert list(o.assign(x)) == [exact_nearest(v, cent) for v in x]


def test_assign_duplicate_centroids_lowest_index():
    cent = np.array([[1, 1], [0, 0], [1, 1], [0, 0]], np.float32)
    o = OracleIVF(2, 4, n_max=10)
    o.set_centroids(cent)
    assert list(o.assign([[1, 1], [0.1, 0], [0.9, 1.0]])) == [0, 1, 0]


@pytest.mark.parametrize("P", [1, 3, 9])
def test_probe_matches_exact_rational_order(P):
    rng = np.random.default_rng(11 + P)
    cent = grid_points(rng, 9, 2)
    q = grid_points(rng, 100, 2)
    o = OracleIVF(2, 9, n_max=10)
    o.set_centroids(cent)
    got = o.probe(q, P)
    for r in range(len(q)):
        assert list(got[r]) == exact_probes(q[r], cent, P)


# ------------------------------------------------------------------ search
def _filled(d=8, nlist=12, n=600, seed=3, integer=False, C=8):
    rng = np.random.default_rng(seed)
    if integer:
        cent = grid_points(rng, nlist, d, -3, 3)
        x = grid_points(rng, n, d, -3, 3)
    else:
        cent = rng.standard_normal((nlist, d)).astype(np.float32)
        x = rng.standard_normal((n, d)).astype(np.float32)
    ids = rng.permutation(10 * n)[:n].astype(np.int64)
    o = OracleIVF(d, nlist, C, n_max=10 * n, n_slabs=10 * n)
    o.set_centroids(cent)
    o.add(ids, x)
    return o, cent, x, ids, rng


@pytest.mark.parametrize("integer", [False, True])
def test_full_probe_equals_brute_force(integer):
    """nprobe = nlist scans every list: IVF search is exact kNN."""
    o, cent, x, ids, rng = _filled(integer=integer)
    q = (grid_points(rng, 50, 8, -3, 3) if integer
         else rng.standard_normal((50, 8)).astype(np.float32))
    for k in (1, 7, 30):
        d_o, i_o = o.search(q, k, o.nlist)
        d_b, i_b = brute_knn(q, x, ids, k)
        np.testing.assert_array_equal(i_o, i_b)
        np.testing.assert_allclose(d_o, d_b, rtol=1e-12)
        d_e, i_e = o.exact_knn(q, k)
        np.testing.assert_array_equal(i_e, i_b)


def test_partial_probe_equals_brute_force_over_probed_lists():
    o, cent, x, ids, rng = _filled(seed=5)
    q = rng.standard_normal((40, 8)).astype(np.float32)
    P, k = 3, 10
    d_o, i_o = o.search(q, k, P)
    for r in range(len(q)):
        probed = exact_probes(q[r], cent, P)
        members = np.concatenate([o.list_members(l)[0] for l in probed])
        pos = {int(v): j for j, v in enumerate(ids)}
        xs = x[[pos[int(m)] for m in members]]
        d_b, i_b = brute_knn(q[r:r + 1], xs, members, k)
        np.testing.assert_array_equal(i_o[r], i_b[0])
        np.testing.assert_allclose(d_o[r], d_b[0], rtol=1e-12)


def test_pad_when_fewer_than_k():
    o = OracleIVF(2, 2, 4, n_max=10, n_slabs=10)
    o.set_centroids([[0, 0], [10, 10]])
    o.add([3, 4], [[1, 0], [0, 2]])
    d, i = o.search([[0, 0]], 5, 1)
    assert list(i[0]) == [3, 4, -1, -1, -1]
    assert d[0, 0] == 1 and d[0, 1] == 4 and np.isinf(d[0, 2:]).all()


def test_ties_in_topk_go_to_lower_id():
    o = OracleIVF(1, 1, 4, n_max=100, n_slabs=10)
    o.set_centroids([[0]])
    o.add([50, 7, 9, 3], [[2], [-2], [1], [-1]])
    d, i = o.search([[0]], 3, 1)
    assert list(i[0]) == [3, 9, 7] and list(d[0]) == [1, 1, 4]


def test_search_with_probes_matches_search():
    o, cent, x, ids, rng = _filled(seed=9)
    q = rng.standard_normal((30, 8)).astype(np.float32)
    pr = o.probe(q, 4)
    a = o.search(q, 6, 4)
    b = o.search_with_probes(q, 6, pr)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[0], b[0])


def test_golden_tiny_1d():
    """Hand-worked example of tests/golden/tiny_1d.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_1d.txt")
    sec, data = None, {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("["):
            sec = line.strip("[]")
            data[sec] = []
            continue
        data[sec].append([float(t) for t in line.split()])
    cent = np.array(data["centroids"], np.float32)
    pts = data["points"]
    o = OracleIVF(1, len(cent), 2, n_max=100, n_slabs=100)
    o.set_centroids(cent)
    ids = np.array([int(p[0]) for p in pts])
    x = np.array([[p[1]] for p in pts], np.float32)
    o.add(ids, x)
    for p in pts:
        assert o.list_of(int(p[0])) == int(p[2])
    for row in data["search"]:
        qv, k, P = row[0], int(row[1]), int(row[2])
        want_ids = [int(v) for v in row[3:3 + k]]
        want_d = row[3 + k:3 + 2 * k]
        d, i = o.search([[qv]], k, P)
        assert list(i[0]) == want_ids
        assert list(d[0]) == want_d


# ---------------------------------------------- add / remove semantics
class SetModel:
    """Plain dictionary model of the add / remove semantics."""

    def __init__(self):
        self.vec = {}

    def add(self, ids, x):
        for i, v in zip(ids, x):     # later occurrences overwrite earlier
            self.vec[int(i)] = v

    def remove(self, ids):
        n = 0
        for i in ids:
            if int(i) in self.vec:
                del self.vec[int(i)]
                n += 1
        return n


def test_random_ops_match_set_model_and_invariants():
    rng = np.random.default_rng(21)
    d, L, C, nmax = 4, 7, 4, 120
    cent = grid_points(rng, L, d, -2, 2)
    o = OracleIVF(d, L, C, n_max=nmax, n_slabs=1000)
    o.set_centroids(cent)
    m = SetModel()
    for step in range(60):
        if rng.random() < 0.6:
            n = int(rng.integers(0, 25))
            ids = rng.integers(0, nmax, size=n)     # duplicates + overwrites
            x = grid_points(rng, n, d, -2, 2)
            got = o.add(ids, x)
            assert got == len(set(ids.tolist()))
            m.add(ids, x)
        else:
            n = int(rng.integers(0, 25))
            ids = rng.integers(0, nmax, size=n)
            assert o.remove(ids) == m.remove(ids)
        assert o.ntotal == len(m.vec)
        seen = []
        used = 0
        for l in range(L):
            mids, seq, slot = o.list_members(l)
            seen += mids.tolist()
            fill, live = o.list_slabs(l)
            used += len(fill)
            # every slab but the head is full; live counts match members
            assert (fill[:-1] == C).all() if len(fill) else True
            assert (live >= 1).all() and live.sum() == len(mids)
            assert np.bincount(seq, minlength=len(fill)).tolist() == live.tolist()
            pairs = set(zip(seq.tolist(), slot.tolist()))
            assert len(pairs) == len(mids)                 # no slot twice
            assert all(s < fill[q] for q, s in zip(seq, slot))
            xs = o.list_vectors(l)
            for i, v in zip(mids, xs):
                np.testing.assert_array_equal(v, m.vec[int(i)])
                assert exact_nearest(v, cent) == l
        assert sorted(seen) == sorted(m.vec)              # each id once
        assert used + o.free_slabs == 1000


def test_duplicate_in_batch_last_wins():
    o = OracleIVF(1, 2, 4, n_max=10, n_slabs=10)
    o.set_centroids([[0], [10]])
    assert o.add([5, 5, 6], [[0.5], [9.5], [1]]) == 2
    assert o.list_of(5) == 1 and o.list_of(6) == 0
    assert list(o.list_members(0)[0]) == [6]


def test_overwrite_is_delete_then_insert():
    o = OracleIVF(1, 2, 4, n_max=10, n_slabs=10)
    o.set_centroids([[0], [10]])
    o.add([1, 2, 3], [[0], [1], [2]])
    o.add([2], [[11]])
    assert list(o.list_members(0)[0]) == [1, 3]
    assert list(o.list_members(1)[0]) == [2]
    d, i = o.search([[1]], 3, 2)
    assert list(i[0]) == [1, 3, 2] and list(d[0]) == [1, 1, 100]


def test_remove_idempotent_and_absent_ids():
    o, cent, x, ids, rng = _filled(seed=13)
    n0 = o.ntotal
    drop = ids[:100]
    assert o.remove(np.concatenate([drop, drop])) == 100
    assert o.remove(drop) == 0
    assert o.ntotal == n0 - 100
    q = rng.standard_normal((20, 8)).astype(np.float32)
    _, i = o.search(q, 50, o.nlist)
    assert not set(i.ravel().tolist()) & set(drop.tolist())


def test_out_of_range_ids_rejected_without_change():
    o = OracleIVF(1, 1, 4, n_max=10, n_slabs=10)
    o.set_centroids([[0]])
    o.add([1], [[0]])
    with pytest.raises(OracleError) as e:
        o.add([2, 10], [[0], [0]])
    assert e.value.status == oracle.E_ARG and o.ntotal == 1
    with pytest.raises(OracleError):
        o.remove([1, -1])
    assert o.ntotal == 1


def test_untrained_is_state_error():
    o = OracleIVF(1, 1, 4, n_max=10, n_slabs=10)
    with pytest.raises(OracleError) as e:
        o.add([1], [[0]])
    assert e.value.status == oracle.E_STATE


# ------------------------------------------------------ slab bookkeeping
@pytest.mark.parametrize("n,C", [(1, 4), (4, 4), (5, 4), (100, 32), (64, 32)])
def test_slab_count_closed_form(n, C):
    o = OracleIVF(1, 1, C, n_max=1000, n_slabs=1000)
    o.set_centroids([[0]])
    o.add(np.arange(n), np.zeros((n, 1)))
    fill, live = o.list_slabs(0)
    nsl = -(-n // C)
    assert len(fill) == nsl and o.free_slabs == 1000 - nsl
    want = [C] * (nsl - 1) + [n - C * (nsl - 1)]
    assert fill.tolist() == want and live.tolist() == want


def test_delete_all_returns_every_slab():
    o, *_ = _filled(seed=17)
    ids = np.arange(o.n_max)
    o.remove(ids)
    assert o.ntotal == 0 and o.free_slabs == o.n_slabs
    for l in range(o.nlist):
        assert len(o.list_slabs(l)[0]) == 0


def test_sliding_window_frees_oldest_slab():
    C = 8
    o = OracleIVF(1, 1, C, n_max=1000, n_slabs=100)
    o.set_centroids([[0]])
    o.add(np.arange(40), np.zeros((40, 1)))          # 5 full slabs
    free0 = o.free_slabs
    o.remove(np.arange(7))                           # oldest slab: 1 live
    assert o.free_slabs == free0
    o.remove([7])                                    # now empty -> pool
    assert o.free_slabs == free0 + 1
    for step in range(10):                           # steady window
        base = 40 + C * step
        o.add(np.arange(base, base + C), np.zeros((C, 1)))
        o.remove(np.arange(base - 32, base - 32 + C))
        assert o.free_slabs == free0 + 1


def test_admission_is_all_or_nothing():
    C = 4
    o = OracleIVF(1, 2, C, n_max=100, n_slabs=3)
    o.set_centroids([[0], [10]])
    o.add([0, 1, 2], [[0], [0], [0]])                # list 0: fill 3/4
    # list 0 needs ceil((6-1)/4) = 2 more slabs, list 1 needs 1: 3 > 2 free
    with pytest.raises(OracleError) as e:
        o.add(range(10, 17), [[0]] * 6 + [[10]])
    assert e.value.status == oracle.E_NOMEM
    assert o.ntotal == 3 and o.free_slabs == 2
    o.add(range(10, 15), [[0]] * 5)                  # needs exactly 1
    assert o.free_slabs == 1 and o.ntotal == 8


def test_directory_capacity_limits_a_list():
    o = OracleIVF(1, 2, 2, n_max=100, n_slabs=50, dir_cap=3)
    o.set_centroids([[0], [10]])
    o.add(range(6), [[0]] * 6)                       # 3 slabs in list 0
    with pytest.raises(OracleError) as e:
        o.add([20], [[0]])
    assert e.value.status == oracle.E_NOMEM
    o.add([21], [[10]])                              # list 1 still fine


# ------------------------------------------------------------ encodings
def test_bf16_matches_torch_rne():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32) * 1e3,
        np.array([0.0, -0.0, 1.0, -1.5, 3.0e38, -3.4e38, 1e-40, np.inf,
                  -np.inf], np.float32),
        # exact halfway cases, both parities
        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 2.0 + 2 ** -7],
                 np.float32)])
    got = oracle.to_bf16(x)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy()
    np.testing.assert_array_equal(got, want.view(np.uint16))
    back = oracle.from_bf16(got)
    np.testing.assert_array_equal(
        back, torch.from_numpy(x).to(torch.bfloat16).float().numpy())


def test_e4m3_matches_torch_in_range_and_saturates():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.uniform(-440, 440, 20000), rng.standard_normal(20000),
        rng.standard_normal(2000) * 1e-2,
        # halfway points between neighbouring codes
        [1.0625, 1.1875, 17.0, 0.001953125 * 1.5, 2 ** -10]]).astype(np.float32)
    got = oracle.to_e4m3(x, 1.0)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(got, want)
    big = np.array([448.0, 500.0, 1e6, -1e9], np.float32)
    assert oracle.to_e4m3(big, 1.0).tolist() == [0x7e, 0x7e, 0x7e, 0xfe]
    # scaling: v = fl32(x * inv_scale)
    y = rng.standard_normal(1000).astype(np.float32) * 300
    inv = np.float32(1.0 / 0.75)
    np.testing.assert_array_equal(oracle.to_e4m3(y, inv),
                                  oracle.to_e4m3((y * inv).astype(np.float32), 1.0))


def test_e4m3_decode_all_codes_matches_torch():
    torch = pytest.importorskip("torch")
    codes = np.array([c for c in range(256) if c not in (0x7f, 0xff)], np.uint8)
    got = oracle.from_e4m3(codes)
    want = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy()
    np.testing.assert_array_equal(got, want)
    assert got.max() == 448.0 and got[got > 0].min() == 2.0 ** -9


# ------------------------------------------------- distance functions
@pytest.mark.parametrize("n,d,denom", [(1, 1, 1), (5, 3, 1), (17, 8, 4), (40, 33, 16)])
def test_dists_equal_exact_rational_sums(n, d, denom):
    """The FP64 distances every re-rank check compares against: on integer
    and dyadic rows each term and each partial sum is exact in FP64, so the
    result must equal the rational sum exactly, row by row (several n and d,
    so a stride or row-offset mistake shows)."""
    rng = np.random.default_rng(900 + d)
    q = grid_points(rng, 1, d, -60, 60, denom)[0]
    x = grid_points(rng, n, d, -60, 60, denom)
    got = oracle.dists(q, x)
    want = [float(exact_sq(q, row)) for row in x]
    assert got.tolist() == want


def test_dists_hand_value():
    """The rows (1, 2, 2) and (4, -2, 2) from the origin: 1 + 4 + 4 = 9 and
    16 + 4 + 4 = 24; from (1, 0, 1): 0 + 4 + 1 = 5 and 9 + 4 + 1 = 14."""
    got = oracle.dists([0, 0, 0], [[1, 2, 2], [4, -2, 2]])
    assert got.tolist() == [9.0, 24.0]
    got = oracle.dists([1, 0, 1], [[1, 2, 2], [4, -2, 2]])
    assert got.tolist() == [5.0, 14.0]


def test_approx_bf16_exact_inputs_equal_the_distance():
    """Integers of magnitude <= 256 are exact in bfloat16, so the expanded
    form ||q||^2 + ||x||^2 - 2 q^.x^ equals the exact squared distance."""
    rng = np.random.default_rng(31)
    for n, d in [(1, 4), (9, 16), (33, 96)]:
        q = rng.integers(-256, 257, size=d).astype(np.float32)
        x = rng.integers(-256, 257, size=(n, d)).astype(np.float32)
        got, mag = oracle.approx_dists(q, x, "bf16")
        want = [float(exact_sq(q, row)) for row in x]
        assert got.tolist() == want
        assert (mag >= got).all()


def test_approx_bf16_hand_value():
    """q = (257), x = (3): 257 lies halfway between the bfloat16 values 256
    and 258 and rounds to the even one, 256; the norms keep the unrounded
    257, so the value is 257^2 + 3^2 - 2 * 256 * 3 = 64522 (the exact
    distance is 254^2 = 64516)."""
    got, mag = oracle.approx_dists([257.0], [[3.0]], "bf16")
    assert got.tolist() == [64522.0]
    assert mag.tolist() == [257.0 ** 2 + 9 + 2 * 768]


def _e4m3_exact_rows(rng, n, d, lim):
    """Rows of small integers in [-lim, lim]: exact in E4M3 (up to 16) and
    after scaling by 2 or 4 when lim is 8."""
    return rng.integers(-lim, lim + 1, size=(n, d)).astype(np.float64)


@pytest.mark.parametrize("t_l,qmax", [(1.0, 224.0), (4.0, 112.0)])
def test_approx_fp8_exact_codes_equal_the_distance(t_l, qmax):
    """Residual codes with no rounding: the rows' residuals are integers in
    [-8, 8] (times the list scale t_l in {1, 4}: exact E4M3 values), the
    query's residual has largest magnitude qmax, so its own scale is
    448 / (2 qmax) in {1, 2} and its codes are exact too.  The scales then
    cancel and the value is ||(q - c) - (x - c)||^2 = ||q - x||^2 exactly.
    Each row has its own centroid (a residual taken from another row's
    centroid breaks the identity), the scale 2 / 4 cases fail if either
    scale is not undone."""
    rng = np.random.default_rng(int(t_l))
    n, d = 12, 16
    cent = rng.integers(-50, 51, size=(n, d)).astype(np.float64)
    rq = _e4m3_exact_rows(rng, n, d, 8)
    rq[:, 3] = qmax                        # the query's largest residual entry
    # one query q for every row: q = c_i + rq_i must be the same vector, so
    # the rows' centroids are chosen as q - rq_i
    q = rng.integers(-40, 41, size=d).astype(np.float64)
    cent = q[None, :] - rq
    y = _e4m3_exact_rows(rng, n, d, 8)
    x = cent + y
    inv = np.full(n, t_l, np.float32)
    got, _ = oracle.approx_dists(q.astype(np.float32), x.astype(np.float32), "fp8",
                                 inv, cent.astype(np.float32))
    want = [float(exact_sq(q.astype(np.float32), row)) for row in x.astype(np.float32)]
    assert got.tolist() == want


def test_approx_fp8_rounding_against_torch_codes():
    """General residuals: the value equals the expanded form recomputed
    from torch's own float8_e4m3fn casts of the scaled residuals (scales
    computed by hand in float32), within FP64 rounding.  A few residual
    entries are tiny, so their scaled values fall among the subnormal codes,
    where a scale off by a power of two changes the rounding."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    n, d = 7, 24
    q = rng.standard_normal(d).astype(np.float32)
    cent = rng.standard_normal((n, d)).astype(np.float32)
    cent[:, :4] = q[:4] - np.float32([3e-5, 1.1e-4, -7e-5, 2.3e-4])
    x = (cent + 0.3 * rng.standard_normal((n, d))).astype(np.float32)
    x[:, 4:8] = cent[:, 4:8] + np.float32([5e-5, -1.7e-4, 9e-5, 2e-4])
    inv = (448.0 / (2.0 * np.abs(x - cent).max(axis=1))).astype(np.float32)
    got, _ = oracle.approx_dists(q, x, "fp8", inv, cent)
    for i in range(n):
        r = (q - cent[i]).astype(np.float32)
        y = (x[i] - cent[i]).astype(np.float32)
        tq = np.float32(448.0) / (np.float32(2.0) * np.abs(r).max())
        cq = torch.from_numpy((r * tq).astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
        cy = torch.from_numpy((y * inv[i]).astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
        s = 1.0 / (float(inv[i]) * float(tq))
        want = (r.astype(np.float64) ** 2).sum() + (y.astype(np.float64) ** 2).sum() \
            - 2.0 * s * (cq * cy).sum()
        assert abs(got[i] - want) <= 1e-12 * abs(want) + 1e-12


# ------------------------------------------------------ quantizer training
def _golden_splitmix():
    out = {}
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        seed, vals = line.split(":")
        out[int(seed)] = [int(v) for v in vals.split()]
    return out


def test_splitmix64_matches_published_outputs():
    for seed, vals in _golden_splitmix().items():
        np.testing.assert_array_equal(oracle.splitmix64(seed, len(vals)),
                                      np.array(vals, dtype=np.uint64))


def test_kmeans_init_rows_follow_the_generator():
    """Initial rows = SplitMix64 outputs mod n in draw order, repeats
    skipped (checked against the published outputs)."""
    vals = _golden_splitmix()[1234567]
    n = 7
    want = []
    for v in vals:
        if v % n not in want:
            want.append(v % n)
    rows = oracle.kmeans_init_rows(n, len(want), 1234567)
    np.testing.assert_array_equal(rows, want)
    assert len(set(oracle.kmeans_init_rows(1000, 500, 9).tolist())) == 500


def _two_blobs(rng):
    a = rng.integers(-3, 4, (50, 6)) - 100
    b = rng.integers(-3, 4, (70, 6)) + 100
    return np.concatenate([a, b]).astype(np.float32)


def test_kmeans_one_step_is_the_blob_means():
    """Two well-separated integer blobs, initial rows in different blobs:
    one Lloyd step gives the FP32 rounding of each blob's mean."""
    x = _two_blobs(np.random.default_rng(3))
    seed = next(s for s in range(100)
                if len({int(r >= 50) for r in oracle.kmeans_init_rows(len(x), 2, s)}) == 2)
    cent, lab = oracle.kmeans(x, 2, 1, seed)
    first = int(oracle.kmeans_init_rows(len(x), 2, seed)[0] >= 50)
    means = [x[:50].astype(np.float64).mean(0), x[50:].astype(np.float64).mean(0)]
    np.testing.assert_array_equal(cent[0], means[first].astype(np.float32))
    np.testing.assert_array_equal(cent[1], means[1 - first].astype(np.float32))
    assert (lab == np.where(np.arange(len(x)) < 50, first, 1 - first)).all()


def test_kmeans_empty_cell_keeps_its_centroid():
    """98 copies of A and 2 of B; when both initial rows are copies of A the
    two centroids tie, every row goes to the lower index, and the other
    centroid keeps its value A."""
    A = np.arange(4, dtype=np.float32)
    B = A + 8
    x = np.stack([A] * 98 + [B] * 2)
    seed = next(s for s in range(1000) if (oracle.kmeans_init_rows(100, 2, s) < 98).all())
    cent, lab = oracle.kmeans(x, 2, 1, seed)
    np.testing.assert_array_equal(cent[1], A)
    np.testing.assert_array_equal(cent[0], ((98 * A.astype(np.float64) + 2 * B) / 100).astype(np.float32))
    # final assignment: A lies on centroid 1, B is nearer the shifted centroid 0
    assert (lab[:98] == 1).all() and (lab[98:] == 0).all()


def _objective(x, cent):
    d = np.stack([oracle.dists(c, x) for c in cent])   # FP64 distances
    return d.min(axis=0).sum()


def test_kmeans_objective_never_increases_and_fixed_point():
    rng = np.random.default_rng(11)
    ctr = rng.uniform(-1, 1, (12, 8))
    x = (ctr[rng.integers(0, 12, 3000)] + 0.2 * rng.standard_normal((3000, 8))).astype(np.float32)
    js = [_objective(x, oracle.kmeans(x, 12, it, 5)[0]) for it in range(0, 8)]
    assert all(js[i + 1] <= js[i] * (1 + 1e-12) for i in range(len(js) - 1)), js
    # converged: another step changes nothing, and each centroid is the
    # FP32 mean of its rows
    c1, lab = oracle.kmeans(x, 12, 60, 5)
    c2, _ = oracle.kmeans(x, 12, 61, 5)
    np.testing.assert_array_equal(c1, c2)
    for k in range(12):
        sel = x[lab == k].astype(np.float64)
        if len(sel):
            np.testing.assert_allclose(c1[k], sel.mean(0), rtol=1e-6, atol=1e-6)


def test_fp8_list_scales_closed_form():
    """s_l = 448 / R_l with R_l the distance to the nearest other centroid;
    one list alone falls back to 448 / (2 max_j |c_j|)."""
    c = np.zeros((3, 4), np.float32)
    c[1, 0] = 3.0
    c[2, 1] = 4.0
    np.testing.assert_array_equal(oracle.fp8_list_scales(c),
                                  np.float32([448 / 3, 448 / 3, 448 / 4]))
    one = np.array([[1.0, -2.5, 0.5, 2.0]], np.float32)
    np.testing.assert_array_equal(oracle.fp8_list_scales(one), np.float32([448 / 5]))
    np.testing.assert_array_equal(oracle.fp8_list_scales(np.zeros((1, 4), np.float32)),
                                  np.float32([1.0]))


# ------------------------------------------------------------ compaction
def _one_list(C=4, n=10):
    o = OracleIVF(2, 1, slab_size=C, n_max=64, n_slabs=16)
    o.set_centroids(np.zeros((1, 2), np.float32))
    o.add(np.arange(n), np.arange(2 * n, dtype=np.float32).reshape(n, 2))
    return o


def test_compact_worked_example():
    """C = 4, ids 0..9 appended in order (slabs [0 1 2 3] [4 5 6 7] [8 9]);
    deleting 0, 1, 2, 5, 8 leaves 5 live members in 3 slabs.  Compaction
    rewrites them densely in member order -- 3 4 6 7 in slab 0, 9 in slab 1
    -- and returns slab 2 to the pool; the next insert lands in slab 1,
    slot 1."""
    o = _one_list()
    o.remove([0, 1, 2, 5, 8])
    free0 = o.free_slabs
    assert [x.tolist() for x in o.list_slabs(0)] == [[4, 4, 2], [1, 3, 1]]
    assert o.compact(min_free=1) == (1, 5)
    ids, seq, slot = o.list_members(0)
    assert ids.tolist() == [3, 4, 6, 7, 9]
    assert seq.tolist() == [0, 0, 0, 0, 1]
    assert slot.tolist() == [0, 1, 2, 3, 0]
    assert [x.tolist() for x in o.list_slabs(0)] == [[4, 1], [4, 1]]
    assert o.free_slabs == free0 + 1
    o.add([10], [[0.5, 0.5]])
    ids, seq, slot = o.list_members(0)
    assert (ids[-1], seq[-1], slot[-1]) == (10, 1, 1)
    assert [x.tolist() for x in o.list_slabs(0)] == [[4, 2], [4, 2]]
    # nothing left to free: a second pass is a no-op
    assert o.compact(min_free=1) == (0, 0)


def test_compact_min_free_and_budget_rules():
    """A list is compacted only when it frees at least min_free slabs; lists
    are taken in index order until the next one would pass max_moves."""
    o = OracleIVF(1, 2, slab_size=4, n_max=64, n_slabs=32)
    o.set_centroids(np.array([[0.0], [100.0]], np.float32))
    o.add(np.arange(16), np.zeros((16, 1), np.float32))            # list 0: 4 slabs
    o.add(np.arange(16, 32), np.full((16, 1), 100.0, np.float32))  # list 1: 4 slabs
    o.remove([1, 2, 3, 5, 6, 7])          # list 0: 10 live -> 3 slabs, frees 1
    o.remove([16, 17, 18, 20, 21, 22, 24, 25, 26])  # list 1: 7 live -> 2 slabs, frees 2
    assert o.compact(min_free=3) == (0, 0)
    assert o.compact(min_free=2, max_moves=6) == (0, 0)       # list 1 alone needs 7
    assert o.compact(min_free=1, max_moves=9) == (0, 0)       # list 0 (10) ends the pass
    assert o.compact(min_free=1, max_moves=16) == (1, 10)     # list 0 only
    assert [len(x) for x in o.list_slabs(0)] == [3, 3]
    assert o.compact(min_free=1, max_moves=7) == (2, 7)       # then list 1
    assert [x.tolist() for x in o.list_slabs(1)] == [[4, 3], [4, 3]]
    with pytest.raises(OracleError):
        o.compact(min_free=0)


def test_compact_keeps_search_and_members():
    """Random inserts and deletes, then compaction: every list's members keep
    their order and become dense, the freed slab count is the sum over lists
    of (slabs - ceil(n / C)), and every search returns the same result."""
    rng = np.random.default_rng(7)
    d, L, C = 8, 6, 8
    cent = rng.standard_normal((L, d)).astype(np.float32)
    o = OracleIVF(d, L, slab_size=C, n_max=4000, n_slabs=800)
    o.set_centroids(cent)
    x = (cent[rng.integers(0, L, 3000)] + 0.3 * rng.standard_normal((3000, d))).astype(np.float32)
    o.add(np.arange(3000), x)
    o.remove(rng.choice(3000, 1900, replace=False))
    q = rng.standard_normal((40, d)).astype(np.float32)
    before = [o.search(q, 7, P) for P in (1, 3, L)]
    members = [o.list_members(l)[0].copy() for l in range(L)]
    before_slabs = [o.list_slabs(l)[0].copy() for l in range(L)]
    expect = sum(len(o.list_slabs(l)[0]) - (o.list_size(l) + C - 1) // C for l in range(L))
    free0 = o.free_slabs
    freed, moved = o.compact(min_free=1)
    assert freed == expect > 0 and o.free_slabs == free0 + freed
    fragmented = [l for l in range(L)
                  if len(o.list_slabs(l)[0]) < len(before_slabs[l])]
    assert moved == sum(o.list_size(l) for l in fragmented)
    for l in range(L):
        ids, seq, slot = o.list_members(l)
        np.testing.assert_array_equal(ids, members[l])
        j = np.arange(len(ids))
        np.testing.assert_array_equal(seq, j // C)
        np.testing.assert_array_equal(slot, j % C)
    for (bd, bi), P in zip(before, (1, 3, L)):
        ad, ai = o.search(q, 7, P)
        np.testing.assert_array_equal(ad, bd)
        np.testing.assert_array_equal(ai, bi)
