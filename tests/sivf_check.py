"""Helpers shared by the tests: build/load of the CUDA library, the
invariant checker of the device bookkeeping, and the comparisons of device
results with the oracle."""
from __future__ import annotations

import os
import re

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols() -> list[str]:
    """Every function include/sivf.h declares."""
    src = open(os.path.join(ROOT, "include", "sivf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sivf_[a-z_0-9]+)\s*\(", src)))


def build_lib():
    from paper_2601_11808_gb300 import build, sivf
    build.build()
    return sivf.load()


# ------------------------------------------------------------- state checks
def device_lists(dump: dict, C: int):
    """Per list: slab sequence and members (id, slab position, slot) in
    directory order, from a device dump."""
    out = []
    for l, n in enumerate(dump["list_nslabs"]):
        slabs = dump["list_dir"][l, :n]
        ids, seq, slot = [], [], []
        for p, s in enumerate(slabs):
            bits = dump["slab_bits"][s]
            for o in range(C):
                if (int(bits[o >> 5]) >> (o & 31)) & 1:
                    ids.append(int(dump["slab_ids"][s, o]))
                    seq.append(p)
                    slot.append(o)
        out.append((slabs, np.array(ids, np.int64), np.array(seq), np.array(slot)))
    return out


def check_invariants(dump: dict, C: int, n_slabs: int):
    """Consistency of the device bookkeeping on its own (Theorems 1-3 and
    the slab accounting): every live id exactly once, the address table
    agrees with the slots, live counts equal bit counts, free + used = S,
    free slabs are clean, heads are the last slab of their list."""
    meta, bits, att = dump["slab_meta"], dump["slab_bits"], dump["att"]
    lists = device_lists(dump, C)
    used = set()
    live_ids = []
    for l, (slabs, ids, seq, slot) in enumerate(lists):
        for s in slabs:
            assert 0 <= s < n_slabs, f"slab {s} out of range"
            assert s not in used, f"slab {s} in two lists"
            used.add(int(s))
            lst, fill, live = meta[s]
            assert lst == l, f"slab {s} owned by {lst}, listed in {l}"
            pop = sum(bin(int(w)).count("1") for w in bits[s])
            assert pop == live, f"slab {s}: live {live} != popcount {pop}"
            assert 1 <= live <= fill <= C
            # no bit at or beyond fill
            for o in range(fill, C):
                assert not (int(bits[s][o >> 5]) >> (o & 31)) & 1
        if len(slabs) > 1:
            assert all(meta[s][1] == C for s in slabs[:-1]), f"list {l}: non-head slab not full"
        h = dump["list_head"][l]
        assert h == -1 or (len(slabs) and h == slabs[-1]), f"list {l}: head {h}"
        if h == -1 and len(slabs):
            assert meta[slabs[-1]][1] == C
        for i, p, o in zip(ids, seq, slot):
            s = slabs[p]
            assert att[i] == (int(s) << 32) | int(o), f"att of id {i}"
        live_ids += ids.tolist()
    assert len(live_ids) == len(set(live_ids)), "an id is live twice"
    live_set = set(live_ids)
    valid = np.nonzero(att >= 0)[0]
    assert set(valid.tolist()) == live_set, "address table has stale entries"
    free = dump["free_stack"]
    assert len(free) == dump["n_free"]
    assert len(set(free.tolist())) == len(free)
    assert not (set(free.tolist()) & used)
    assert len(free) + len(used) == n_slabs
    for s in free:
        assert tuple(meta[s]) == (-1, 0, 0) and not bits[s].any()
    return lists


def compare_state(dump: dict, orc, C: int, n_slabs: int):
    """Device bookkeeping equals the oracle: same members per list in the same
    order, same slab positions and slots, same slab fill/live sequence,
    same number of free slabs."""
    lists = check_invariants(dump, C, n_slabs)
    assert dump["n_free"] == orc.free_slabs
    for l, (slabs, ids, seq, slot) in enumerate(lists):
        o_ids, o_seq, o_slot = orc.list_members(l)
        np.testing.assert_array_equal(ids, o_ids, err_msg=f"list {l} members")
        np.testing.assert_array_equal(seq, o_seq, err_msg=f"list {l} slab positions")
        np.testing.assert_array_equal(slot, o_slot, err_msg=f"list {l} slots")
        fill, live = orc.list_slabs(l)
        np.testing.assert_array_equal(dump["slab_meta"][slabs, 1], fill)
        np.testing.assert_array_equal(dump["slab_meta"][slabs, 2], live)


# ------------------------------------------------------------ search checks
def compare_topk(gd, gi, od, oi, rtol: float = 1e-5, what: str = ""):
    """Device top-k (float32) against oracle top-k (float64).

    Rank by rank the distances agree within `rtol` (relative).  The id sets
    agree except for ids whose distance lies within `rtol` of the k-th
    oracle distance (ties at the cut).  Padding is (+inf, -1) on both.
    Returns the number of queries whose id sets differed at a tie."""
    gd = np.asarray(gd, np.float64)
    od = np.asarray(od, np.float64)
    gi, oi = np.asarray(gi), np.asarray(oi)
    nq, k = od.shape
    ties = 0
    for r in range(nq):
        fin = np.isfinite(od[r])
        assert (np.isfinite(gd[r]) == fin).all(), f"{what} q{r}: padding differs"
        assert (gi[r][~fin] == -1).all()
        err = np.abs(gd[r][fin] - od[r][fin])
        tol = rtol * np.maximum(od[r][fin], 1e-30) + 1e-30
        assert (err <= tol).all(), (
            f"{what} q{r}: distance error {np.max(err / np.maximum(od[r][fin], 1e-30)):.3g}")
        sg, so = set(gi[r][fin].tolist()), set(oi[r][fin].tolist())
        if sg != so:
            cut = od[r][fin][-1]
            band = cut * (1 - 2 * rtol)
            g_extra = [d for d, i in zip(gd[r], gi[r]) if i in sg - so]
            o_extra = [d for d, i in zip(od[r], oi[r]) if i in so - sg]
            assert all(d >= band for d in g_extra + o_extra), (
                f"{what} q{r}: id sets differ away from the k-th distance")
            ties += 1
        # within equal distances the order is by id
        for j in range(1, int(fin.sum())):
            if gd[r][j] == gd[r][j - 1]:
                assert gi[r][j] > gi[r][j - 1]
    return ties


# ------------------------------------------- reduced-precision candidates
def approx_oracle(q, xs, dtype, inv_l, cent_l):
    """The oracle's approximate distance of the reduced-precision scan
    (``oracle.approx_dists``) and the bound of an FP32 accumulation of it:
    (FP64 value, norms + 2 s sum |products|)."""
    return oracle.approx_dists(q, xs, dtype, inv_l, cent_l)


# ------------------------------------------------ device index beside oracle
def cuda(t, a, dtype=None):
    x = t.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        x = x.to(dtype)
    return x.cuda()


class Pair:
    """A device index and an oracle driven with the same operations."""

    def __init__(self, torch, d, nlist, C, n_max, n_slabs, cent, dir_cap=0, dtypes=()):
        from paper_2601_11808_gb300.sivf import Index
        self.t = torch
        self.g = Index(d, nlist, C, n_max, n_slabs, dir_cap, dtypes)
        self.o = oracle.OracleIVF(d, nlist, C, n_max, n_slabs, dir_cap or n_slabs)
        self.C, self.S = C, n_slabs
        self.g.set_centroids(cuda(torch, cent))
        self.o.set_centroids(cent)

    def add(self, ids, x):
        from paper_2601_11808_gb300.sivf import SivfError
        try:
            og = self.o.add(ids, x)
            ost = 0
        except oracle.OracleError as e:
            og, ost = 0, e.status
        try:
            gg = self.g.add(cuda(self.t, np.asarray(ids, np.int64)),
                            cuda(self.t, np.asarray(x, np.float32).reshape(-1, self.g.d)),
                            sync=True)
            gst = 0
        except SivfError as e:
            gg, gst = 0, e.status
        assert (gst, gg) == (ost, og), f"add status/count {gst, gg} != oracle {ost, og}"
        return gst

    def remove(self, ids):
        from paper_2601_11808_gb300.sivf import SivfError
        try:
            og, ost = self.o.remove(ids), 0
        except oracle.OracleError as e:
            og, ost = 0, e.status
        try:
            gg = self.g.remove(cuda(self.t, np.asarray(ids, np.int64)), sync=True)
            gst = 0
        except SivfError as e:
            gg, gst = 0, e.status
        assert (gst, gg) == (ost, og), f"remove status/count {gst, gg} != oracle {ost, og}"
        return gst

    def compact(self, min_free=1, max_moves=1 << 40):
        og = self.o.compact(min_free, max_moves)
        gg = self.g.compact(min_free, max_moves, sync=True)
        assert gg == og, f"compact (freed, moved) {gg} != oracle {og}"
        return gg

    def check(self):
        compare_state(self.g.dump(), self.o, self.C, self.S)
        assert self.g.stats()["ntotal"] == self.o.ntotal
        np.testing.assert_array_equal(
            self.g.list_sizes(), [self.o.list_size(l) for l in range(self.g.nlist)])

    def search(self, q, k, P):
        gd, gi = self.g.search(cuda(self.t, q), k, P)
        od, oi = self.o.search(q, k, P)
        return gd.cpu().numpy(), gi.cpu().numpy(), od, oi


# ------------------------------------------------- space model and merge
def slab_header_overhead(d: int, slab_size: int = 32, header_bytes: int = 128,
                         payload_bytes: int = 4) -> float:
    """Fraction of slab memory spent on the per-slab header: the space model
    of Sec. 3.5.3 (metadata amortised over C vectors of d floats)."""
    return header_bytes / (slab_size * d * payload_bytes)


def merge_topk_host(dists, ids, k: int):
    """Merge per-shard top-k lists (shape [shards, nq, k']) into one top-k by
    (distance, id), the gather step of the paper's scatter-gather search
    (Sec. 4.2).  Padding (+inf, -1) sorts last."""
    d = np.concatenate(list(dists), axis=1)
    i = np.concatenate(list(ids), axis=1)
    key_i = np.where(i < 0, np.iinfo(np.int64).max, i)
    out_d = np.empty((d.shape[0], k), d.dtype)
    out_i = np.empty((d.shape[0], k), np.int64)
    for r in range(d.shape[0]):
        order = np.lexsort((key_i[r], d[r]))[:k]
        out_d[r] = d[r][order]
        out_i[r] = i[r][order]
    return out_d, out_i
