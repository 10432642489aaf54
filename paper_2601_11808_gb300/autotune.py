"""Scan-tile autotuning with an on-disk cache, and a slab-size chooser.

The list scan's work split (queries per tile, slabs per chunk, work items per
SM, k-select width, nearest-list-first) is held per batch-shape bucket in the
index; ``sivf_autotune`` times one batch shape over a set of tiles and
installs the fastest.  This module runs it for every bucket a workload's
batches fall in and keeps the results in a JSON file keyed by the GPU name and
the index shape, so a later process installs them without timing again.

``pick_slab_size`` is the one choice made before an index exists: it builds
a trial index for each candidate slab size from a sample of the data, tunes
its tiles and times the same searches.
"""
from __future__ import annotations

import json
import math
import os

from . import sivf

DTYPE_NAMES = {sivf.FP32: "fp32", sivf.BF16: "bf16", sivf.FP8E4M3: "fp8"}


def bucket(nlist: int, nq: int, k: int, nprobe: int, dtype: str) -> str:
    """The table bucket a search falls in (the same rule as the library's)."""
    r = max(nq * nprobe / nlist, 1.0 / 256)
    b = min(max(int(math.floor(math.log2(r))) + 8, 0), 23)
    kept = k if dtype == "fp32" else 4 * k
    kb = 0 if kept <= 16 else 1 if kept <= 64 else 2 if kept <= 256 else 3
    return f"{dtype}/{b}/{kb}"


def _key(index: sivf.Index, device_name: str) -> str:
    return (f"{device_name}|d{index.d}|L{index.nlist}|C{index.slab_size}|"
            f"{','.join(index.scan_dtypes) or 'fp32'}")


def load_cache(path: str) -> dict:
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(path: str, cache: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(index: sivf.Index, queries, shapes, cache_path: str | None = None, reps: int = 3,
         retune: bool = False) -> dict:
    """Install tuned tiles for every (nq, k, nprobe, dtype) in `shapes`.

    `queries` is a CUDA float32 tensor with at least max(nq) rows; the
    first nq rows stand for a batch of that size.  Shapes that fall in the
    same bucket are tuned once.  Returns {bucket: {"tile": ..., "ms": ...}}
    for the buckets seen."""
    import torch
    dev = torch.cuda.get_device_name(queries.device)
    cache = load_cache(cache_path) if cache_path else {}
    entry = cache.setdefault(_key(index, dev), {})
    seen = {}
    for nq, k, nprobe, dtype in shapes:
        b = bucket(index.nlist, nq, k, nprobe, dtype)
        if b in seen:
            continue
        if b in entry and not retune:
            index.set_tile(dtype, nq, k, nprobe, entry[b]["tile"])
            seen[b] = entry[b]
            continue
        tile, ms = index.autotune(queries[:nq].contiguous(), k, nprobe, dtype, reps)
        entry[b] = {"tile": tile, "ms": ms, "shape": [int(nq), int(k), int(nprobe)]}
        seen[b] = entry[b]
    if cache_path:
        save_cache(cache_path, cache)
    return seen


def pick_slab_size(d: int, nlist: int, x, ids, centroids, queries, k: int, nprobe: int,
                   dtype: str = "fp32", sizes=(32, 64, 128), reps: int = 5) -> dict:
    """Time the same search on trial indexes holding `x` (CUDA float32 [n, d])
    at each slab size; returns {"best": C, "ms": {C: ms}}.  Each trial gets
    its own tuned tile for the batch."""
    import torch
    n = x.shape[0]
    out = {}
    for C in sizes:
        S = 2 * (n // C + nlist)
        dts = () if dtype == "fp32" else (dtype,)
        g = sivf.Index(d, nlist, C, int(ids.max().item()) + 1, S, 0, dts)
        try:
            g.set_centroids(centroids)
            g.add(ids, x)
            g.sync()
            _, ms = g.autotune(queries, k, nprobe, dtype, reps)
            out[C] = ms
        finally:
            g.close()
            torch.cuda.synchronize()
    return {"best": min(out, key=out.get), "ms": out}
