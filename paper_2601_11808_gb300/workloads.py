"""Seeded synthetic inputs shaped like the paper's sliding-window workloads.

This module only draws random numbers; it holds none of the index's
arithmetic.  Both the CUDA path and the CPU oracle take their inputs from
here, so the two always see the same vectors.

Every stream is cut into fixed blocks of ``BLOCK`` vectors and block ``b`` of
stream ``s`` is drawn from ``PCG64(SeedSequence([seed, s, b]))``; a vector's
value therefore depends only on its position in the stream, never on how a
caller batches it.  Streams: 0 = mixture centers, 1 = database vectors,
2 = queries, 3 = extra centroids (sample points, used when there are more
lists than mixture components), 12 = the rank permutation of a Zipf-skewed
mixture (the skewed ingestion workload of the paper's Section 5.4 draws its
components with probability falling as a power of their rank).

The paper's datasets (SIFT1M, GIST1M, Deep1B, T2I-1B, DINO10B) are not
available; these mixtures stand in for them with the same dimensions and
value ranges (SIFT-like: d=128 integers in [0, 255]; Deep-like: d=96, unit
norm).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BLOCK = 4096


@dataclass(frozen=True)
class Workload:
    name: str
    d: int
    n_comp: int          # mixture components
    kind: str            # "uniform_box" | "sift" | "sphere"
    sigma: float
    nlist: int
    slab_size: int
    window: int          # live vectors in the sliding window
    step: int            # vectors inserted (and oldest deleted) per step
    n_queries: int
    k: int
    nprobes: tuple = field(default=(8,))
    seed: int = 0
    zipf: float = 0.0    # > 0: components drawn with P(rank r) ~ r^-zipf


# the workload shapes (sizes, distributions and index parameters)
CONFIGS = {
    "tiny_window": Workload("tiny_window", d=32, n_comp=64, kind="uniform_box",
                            sigma=0.1, nlist=64, slab_size=32, window=20_000,
                            step=2_000, n_queries=200, k=10, nprobes=(8,)),
    "sift_window": Workload("sift_window", d=128, n_comp=1024, kind="sift",
                            sigma=20.0, nlist=1024, slab_size=64,
                            window=1_000_000, step=10_000, n_queries=10_000,
                            k=10, nprobes=(8, 32, 128)),
    "deep_precision": Workload("deep_precision", d=96, n_comp=4096,
                               kind="sphere", sigma=0.02, nlist=4096,
                               slab_size=32, window=10_000_000, step=0,
                               n_queries=10_000, k=100, nprobes=(64,)),
    "mixed_batches": Workload("mixed_batches", d=128, n_comp=64,
                              kind="uniform_box", sigma=0.1, nlist=2048,
                              slab_size=64, window=5_000_000, step=0,
                              n_queries=4096, k=10,
                              nprobes=(8, 16, 32, 64, 128)),
    "serving": Workload("serving", d=128, n_comp=16384, kind="uniform_box",
                        sigma=0.1, nlist=16384, slab_size=128,
                        window=100_000_000, step=0, n_queries=256, k=10,
                        nprobes=(32,)),
    "zipf_ingest": Workload("zipf_ingest", d=128, n_comp=1024, kind="sift",
                            sigma=20.0, nlist=1024, slab_size=64,
                            window=1_000_000, step=0, n_queries=10_000, k=10,
                            nprobes=(8,), zipf=1.0),
}


def _rng(seed: int, stream: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(
        np.random.SeedSequence([int(seed), int(stream), int(block)])))


def centers(w: Workload) -> np.ndarray:
    """Mixture centers, float32 [n_comp, d]."""
    g = _rng(w.seed, 0, 0)
    if w.kind == "uniform_box":
        c = g.uniform(-1.0, 1.0, size=(w.n_comp, w.d))
    elif w.kind == "sift":
        c = g.uniform(0.0, 255.0, size=(w.n_comp, w.d))
    elif w.kind == "sphere":
        c = g.standard_normal(size=(w.n_comp, w.d))
        c /= np.linalg.norm(c, axis=1, keepdims=True)
    else:
        raise ValueError(w.kind)
    return c.astype(np.float32)


def zipf_law(w: Workload):
    """(probabilities by rank, rank -> component) of a skewed mixture: the
    component of rank r (1-based) is drawn with probability r^-s / H(n, s),
    H the generalised harmonic number; which component holds which rank is
    a seeded permutation (stream 12), so the heavy components are spread
    over the space rather than being the first rows of `centers`."""
    r = np.arange(1, w.n_comp + 1, dtype=np.float64)
    p = r ** -float(w.zipf)
    p /= p.sum()
    return p, _rng(w.seed, 12, 0).permutation(w.n_comp)


def _components(w: Workload, g: np.random.Generator, law) -> np.ndarray:
    if law is None:
        return g.integers(0, w.n_comp, size=BLOCK)
    p, perm = law
    return perm[g.choice(w.n_comp, size=BLOCK, p=p)]


def _draw(w: Workload, ctr: np.ndarray, stream: int, start: int,
          n: int) -> np.ndarray:
    out = np.empty((n, w.d), np.float32)
    pos = 0
    law = zipf_law(w) if w.zipf > 0 else None
    b0, b1 = start // BLOCK, (start + n + BLOCK - 1) // BLOCK
    for b in range(b0, b1):
        g = _rng(w.seed, stream, b)
        comp = _components(w, g, law)
        noise = g.standard_normal(size=(BLOCK, w.d))
        blk = ctr[comp].astype(np.float64) + w.sigma * noise
        if w.kind == "sift":
            blk = np.clip(np.rint(blk), 0.0, 255.0)
        elif w.kind == "sphere":
            blk /= np.linalg.norm(blk, axis=1, keepdims=True)
        lo = max(start, b * BLOCK) - b * BLOCK
        hi = min(start + n, (b + 1) * BLOCK) - b * BLOCK
        out[pos:pos + hi - lo] = blk[lo:hi]
        pos += hi - lo
    return out


def vectors(w: Workload, start: int, n: int, ctr: np.ndarray | None = None
            ) -> np.ndarray:
    """Database vectors [start, start+n) of the stream, float32 [n, d]."""
    return _draw(w, centers(w) if ctr is None else ctr, 1, start, n)


def queries(w: Workload, start: int, n: int, ctr: np.ndarray | None = None
            ) -> np.ndarray:
    """Queries [start, start+n) from the same mixture, float32 [n, d]."""
    return _draw(w, centers(w) if ctr is None else ctr, 2, start, n)


def index_centroids(w: Workload, ctr: np.ndarray | None = None) -> np.ndarray:
    """Coarse centroids handed to set_centroids: the mixture centers, then
    (when there are more lists than components) sample points of stream 3."""
    ctr = centers(w) if ctr is None else ctr
    if w.nlist <= w.n_comp:
        return np.ascontiguousarray(ctr[: w.nlist])
    extra = _draw(w, ctr, 3, 0, w.nlist - w.n_comp)
    return np.concatenate([ctr, extra], axis=0)


def stream_ids(start: int, n: int, n_max: int) -> np.ndarray:
    """Dense ids of stream positions [start, start+n): position mod n_max."""
    return (np.arange(start, start + n, dtype=np.int64) % int(n_max))


def small(name: str = "tiny_window", **over) -> Workload:
    """A named workload with some fields overridden (for tests)."""
    base = CONFIGS[name]
    fields = dict(base.__dict__)
    fields.update(over)
    return Workload(**fields)


def log_uniform_sizes(seed: int, stream: int, n: int, hi: int) -> np.ndarray:
    """n batch sizes floor(exp(U[0, ln hi])), clipped to [1, hi]."""
    g = _rng(seed, stream, 0)
    return np.clip(np.floor(np.exp(g.uniform(0.0, np.log(hi), size=n))), 1, hi).astype(np.int64)


def mixed_schedule(n_batches: int = 64, max_query: int = 4096, max_delete: int = 100_000,
                   max_insert: int = 50_000, nprobes=(8, 16, 32, 64, 128), seed: int = 0
                   ) -> list:
    """The uneven batch queue of the mixed-batch workload: n_batches each of
    insert, delete and query batches with log-uniform sizes, interleaved
    1:1:1 (insert, delete, query, insert, ...); every query batch draws its
    own nprobe uniformly from `nprobes`.  Entries are (kind, size, nprobe)."""
    qs = log_uniform_sizes(seed, 4, n_batches, max_query)
    ds = log_uniform_sizes(seed, 5, n_batches, max_delete)
    ins = log_uniform_sizes(seed, 6, n_batches, max_insert)
    ps = _rng(seed, 7, 0).choice(np.asarray(nprobes), size=n_batches)
    out = []
    for i in range(n_batches):
        out.append(("add", int(ins[i]), 0))
        out.append(("remove", int(ds[i]), 0))
        out.append(("search", int(qs[i]), int(ps[i])))
    return out


def sample_ids(seed: int, stream: int, block: int, pool: np.ndarray, n: int) -> np.ndarray:
    """n distinct ids drawn without replacement from `pool` (all of it when
    n >= len(pool))."""
    g = _rng(seed, stream, block)
    if n >= len(pool):
        return g.permutation(pool)
    return g.choice(pool, size=n, replace=False)


# ------------------------------------------------- pooled-noise windows
# A window of 10^8 vectors is too large to draw on the host in a benchmark.
# For it, position i gets a mixture component c_i and a row r_i of a fixed
# pool of standard-normal noise vectors, both drawn per block from stream
# 11, and the vector is fl32(center[c_i] + fl32(sigma * pool[r_i])): two
# IEEE single-precision operations, so any device that composes it the same
# way produces the same bits as `pooled_vectors` here.

def noise_pool(w: Workload, size: int) -> np.ndarray:
    """`size` standard-normal noise vectors, float32 [size, d] (stream 10)."""
    return _rng(w.seed, 10, 0).standard_normal(size=(size, w.d), dtype=np.float32)


def pooled_parts(w: Workload, start: int, n: int, pool_size: int):
    """(component, pool row) of stream positions [start, start + n), int64."""
    comp = np.empty(n, np.int64)
    row = np.empty(n, np.int64)
    pos = 0
    for b in range(start // BLOCK, (start + n + BLOCK - 1) // BLOCK):
        g = _rng(w.seed, 11, b)
        c = g.integers(0, w.n_comp, size=BLOCK)
        r = g.integers(0, pool_size, size=BLOCK)
        lo = max(start, b * BLOCK) - b * BLOCK
        hi = min(start + n, (b + 1) * BLOCK) - b * BLOCK
        comp[pos:pos + hi - lo] = c[lo:hi]
        row[pos:pos + hi - lo] = r[lo:hi]
        pos += hi - lo
    return comp, row


def pooled_vectors(w: Workload, start: int, n: int, ctr: np.ndarray,
                   pool: np.ndarray) -> np.ndarray:
    """Window vectors [start, start + n) of a pooled-noise window, float32."""
    if w.kind != "uniform_box":
        raise ValueError("pooled windows are defined for the uniform-box mixture")
    comp, row = pooled_parts(w, start, n, len(pool))
    return ctr[comp] + pool[row] * np.float32(w.sigma)


def request_stream(n: int, rate_per_s: float, mix=(0.7, 0.1, 0.2), sizes=(10_000, 10_000, 256),
                   seed: int = 0, stream: int = 20):
    """A Poisson request stream of n requests at `rate_per_s`: arrival
    offsets (ns, ascending), kinds (0 insert, 1 delete-oldest, 2 query) drawn
    with probabilities `mix`, and log-uniform sizes up to `sizes[kind]`."""
    g = _rng(seed, stream, 0)
    gaps = g.exponential(1e9 / rate_per_s, size=n)
    t = np.cumsum(gaps).astype(np.int64)
    kind = g.choice(3, size=n, p=np.asarray(mix, np.float64))
    u = g.uniform(0.0, 1.0, size=n)
    hi = np.asarray(sizes, np.float64)[kind]
    size = np.clip(np.floor(np.exp(u * np.log(hi))), 1, hi).astype(np.int64)
    return t, kind, size


def vectors_threaded(w: Workload, start: int, n: int, ctr: np.ndarray | None = None,
                     threads: int = 16, stream: int = 1) -> np.ndarray:
    """`vectors` (stream 1) or `queries` (stream 2) drawn by several threads
    over disjoint position ranges; the result is the same array."""
    from concurrent.futures import ThreadPoolExecutor
    ctr = centers(w) if ctr is None else ctr
    out = np.empty((n, w.d), np.float32)
    step = max(BLOCK, -(-n // (threads * BLOCK)) * BLOCK)

    def part(lo):
        hi = min(n, lo + step)
        out[lo:hi] = _draw(w, ctr, stream, start + lo, hi - lo)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(part, range(0, n, step)))
    return out
