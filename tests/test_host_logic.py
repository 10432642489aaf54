"""CPU tests of the boundary and the host-side logic (no GPU needed)."""
import os

import numpy as np
import pytest

from sivf_check import build_lib, header_symbols


def test_library_builds_loads_and_exports_every_declared_symbol():
    lib = build_lib()
    from paper_2601_11808_gb300 import sivf
    declared = header_symbols()
    assert declared == sorted(sivf.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), f"{name} not exported"
    assert "sm_103a" in sivf.sivf_version()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2601_11808_gb300 import sivf
    with pytest.raises(RuntimeError, match="missing"):
        sivf.load(str(tmp_path / "nope.so"))


def test_create_rejects_bad_config_without_gpu():
    """Argument checks happen before any device work."""
    build_lib()
    from paper_2601_11808_gb300 import sivf
    for bad in [dict(d=3), dict(d=258), dict(d=6), dict(nlist=0), dict(slab_size=48),
                dict(n_max=0), dict(n_slabs=0), dict(scan_dtypes=8)]:
        args = dict(d=32, nlist=8, slab_size=32, n_max=100, n_slabs=10, dir_cap=0,
                    scan_dtypes=0)
        args.update(bad)
        with pytest.raises(sivf.SivfError) as e:
            sivf.sivf_create(**args)
        assert e.value.status == sivf.E_ARG


def test_slab_header_overhead_matches_paper():
    """Sec. 5.6.2 reports 0.77% (d=128) and 0.10% (d=960) for a 128-byte
    header amortised over 32 FP32 vectors."""
    from sivf_check import slab_header_overhead
    assert abs(slab_header_overhead(128) - 0.0077) < 0.0002
    assert abs(slab_header_overhead(960) - 0.0010) < 0.00005


def test_merge_topk_host_ties_and_padding():
    from sivf_check import merge_topk_host
    d = np.array([[[1.0, 3.0, np.inf]], [[1.0, 2.0, 3.0]]])
    i = np.array([[[9, 4, -1]], [[5, 7, 2]]])
    od, oi = merge_topk_host(d, i, 5)
    assert oi[0].tolist() == [5, 9, 7, 2, 4]
    assert od[0].tolist() == [1, 1, 2, 3, 3]


def _shard_worker(rank, world, port, q, x, ids, cent, k, P, out):
    import torch.distributed as dist
    import torch
    from oracle import OracleIVF
    from sivf_check import merge_topk_host
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # round-robin routing of inserts (Sec. 4.2); every shard has the same
    # centroids
    mine = np.arange(len(ids)) % world == rank
    o = OracleIVF(x.shape[1], len(cent), 8, n_max=int(ids.max()) + 1, n_slabs=10000)
    o.set_centroids(cent)
    o.add(ids[mine], x[mine])
    d, i = o.search(q, k, P)
    # broadcast deletes: every shard removes what it owns
    gd = [torch.zeros_like(torch.from_numpy(d)) for _ in range(world)]
    gi = [torch.zeros_like(torch.from_numpy(i)) for _ in range(world)]
    dist.all_gather(gd, torch.from_numpy(d))
    dist.all_gather(gi, torch.from_numpy(i))
    if rank == 0:
        md, mi = merge_topk_host(np.stack([t.numpy() for t in gd]),
                                 np.stack([t.numpy() for t in gi]), k)
        np.save(out + "_d.npy", md)
        np.save(out + "_i.npy", mi)
    dist.destroy_process_group()


def test_sharded_search_equals_unsharded_with_gloo(tmp_path):
    """Scatter-gather over 2 gloo ranks, each an oracle shard with the same
    centroids, merged by (distance, id), equals the unsharded index."""
    import socket
    import torch.multiprocessing as mp
    from oracle import OracleIVF
    rng = np.random.default_rng(4)
    cent = rng.standard_normal((16, 8)).astype(np.float32)
    x = rng.standard_normal((3000, 8)).astype(np.float32)
    ids = rng.permutation(5000)[:3000].astype(np.int64)
    q = rng.standard_normal((40, 8)).astype(np.float32)
    k, P = 10, 4
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = str(tmp_path / "m")
    mp.start_processes(_shard_worker, args=(2, port, q, x, ids, cent, k, P, out),
                       nprocs=2, join=True, start_method="spawn")
    o = OracleIVF(8, 16, 8, n_max=5000, n_slabs=10000)
    o.set_centroids(cent)
    o.add(ids, x)
    d, i = o.search(q, k, P)
    np.testing.assert_array_equal(np.load(out + "_i.npy"), i)
    np.testing.assert_array_equal(np.load(out + "_d.npy"), d)


def _chunk_plan(lcnt, nslabs, tq, chmax, spc, ips):
    """The scan's chunking rule (k_srch_plan), restated: per probed list
    nt = ceil(m / tq) query tiles and c = min(chmax, ns, max(1, ceil(ns /
    target))) slab chunks, target = max(spc, ceil(W / (ips * 152))), W the
    sum of nt * ns; returns (items, output runs)."""
    lcnt, nslabs = np.asarray(lcnt, np.int64), np.asarray(nslabs, np.int64)
    act = (lcnt > 0) & (nslabs > 0)
    nt = (lcnt + tq - 1) // tq
    W = int((nt * nslabs)[act].sum())
    slots = ips * 152
    target = max(spc, -(-W // slots))
    c = np.where(act, np.minimum(np.minimum(chmax, nslabs),
                                 np.maximum(1, -(-nslabs // target))), 0)
    return int((nt * c).sum()), int((lcnt * c).sum())


@pytest.mark.parametrize("shape", ["uniform", "zipf", "one_heavy", "thin"])
def test_chunk_plan_stays_within_scratch_bounds(shape):
    """The scratch of a search is sized from the plan's bounds: per launch at
    most nq*P + L + ips*152 work items and nq*P + tq*ips*152 output runs,
    whatever the list lengths (a heavy list is split, but its extra chunks
    are paid for by the work they cover)."""
    rng = np.random.default_rng({"uniform": 0, "zipf": 1, "one_heavy": 2, "thin": 3}[shape])
    L = 1024
    for trial in range(20):
        if shape == "uniform":
            ns = rng.integers(1, 40, L)
        elif shape == "zipf":
            ns = np.maximum(1, (3000 / np.arange(1, L + 1) ** rng.uniform(0.8, 1.4))).astype(int)
        elif shape == "one_heavy":
            ns = np.ones(L, int)
            ns[rng.integers(L)] = int(rng.integers(1000, 100000))
        else:
            ns = rng.integers(1, 5, L)
        nq, P = int(rng.integers(1, 20000)), int(rng.choice([1, 7, 8, 32, 128]))
        lcnt = np.bincount(rng.integers(0, L, nq * P), minlength=L)
        for tq, ips, spc in ((48, 4, 4), (16, 16, 1), (64, 1, 8)):
            chmax = max(1, min(64, 2048 // P))
            items, runs = _chunk_plan(lcnt, ns, tq, chmax, spc, ips)
            assert items <= nq * P + L + ips * 152
            assert runs <= nq * P + tq * ips * 152
