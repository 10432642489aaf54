"""SIVF oracle -- test infrastructure only.

A plain FP64 CPU model of the streaming IVF-Flat index of arxiv 2601.11808,
written in C (``sivf_oracle.c``) and loaded here with ctypes.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2601_11808_gb300``.

Every function of the C file says which part of the paper it follows; the
readings taken where the paper is silent are listed there too.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sivf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsivf_oracle.so")
_lock = threading.Lock()
_lib = None

OK, E_ARG, E_NOMEM, E_STATE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def load_lib(path: str):
    """Load an oracle shared library at ``path`` and declare its signatures."""
    lib = C.CDLL(path)
    p, i32, i64, f32 = C.c_void_p, C.c_int, C.c_int64, C.c_float
    sig = {
        "oivf_create": (p, [i32, i32, i32, i64, i64, i64]),
        "oivf_destroy": (None, [p]),
        "oivf_set_centroids": (i32, [p, p]),
        "oivf_assign": (i32, [p, p, i64, p]),
        "oivf_probe": (i32, [p, p, i64, i32, p]),
        "oivf_search": (i32, [p, p, i64, i32, i32, p, p]),
        "oivf_search_with_probes": (i32, [p, p, i64, i32, i32, p, p, p]),
        "oivf_exact_knn": (i32, [p, p, i64, i32, p, p]),
        "oivf_add": (i32, [p, p, p, i64, p]),
        "oivf_remove": (i32, [p, p, i64, p]),
        "oivf_compact": (i32, [p, i32, i64, p, p]),
        "oivf_ntotal": (i64, [p]),
        "oivf_free_slabs": (i64, [p]),
        "oivf_list_of": (C.c_int32, [p, i64]),
        "oivf_list_size": (i64, [p, i32]),
        "oivf_list_nslabs": (i64, [p, i32]),
        "oivf_list_members": (None, [p, i32, p, p, p]),
        "oivf_list_vectors": (None, [p, i32, p]),
        "oivf_list_slabs": (None, [p, i32, p, p]),
        "oivf_to_bf16": (None, [p, p, i64]),
        "oivf_from_bf16": (None, [p, p, i64]),
        "oivf_to_e4m3": (None, [p, f32, p, i64]),
        "oivf_from_e4m3": (None, [p, p, i64]),
        "oivf_num_threads": (i32, [i32]),
        "oivf_dists": (None, [p, p, i64, i32, p]),
        "oivf_splitmix64": (None, [C.c_uint64, i64, p]),
        "oivf_kmeans_init_rows": (i32, [i64, i32, C.c_uint64, p]),
        "oivf_kmeans": (i32, [p, i64, i32, i32, i32, C.c_uint64, p, p]),
        "oivf_fp8_list_scales": (None, [p, i32, i32, p]),
        "oivf_approx_dists": (None, [p, p, i64, i32, i32, p, p, p, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_lib(build())
        return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def num_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count of the oracle."""
    return int(_load().oivf_num_threads(int(n)))


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}")
        self.status = status


class OracleIVF:
    """FP64 IVF-Flat with per-list ordered members and a slab-record model.

    ``slab_size`` is the slab capacity C, ``n_slabs`` the slab budget S and
    ``dir_cap`` the most slabs one list may hold; they only drive the
    bookkeeping model and the all-or-nothing admission of ``add``.
    """

    def __init__(self, d: int, nlist: int, slab_size: int = 32,
                 n_max: int = 1 << 20, n_slabs: int = 1 << 20,
                 dir_cap: int | None = None, lib=None):
        self._lib = lib if lib is not None else _load()
        self.d, self.nlist, self.C = int(d), int(nlist), int(slab_size)
        self.n_max, self.n_slabs = int(n_max), int(n_slabs)
        self.dir_cap = int(dir_cap if dir_cap is not None else n_slabs)
        self._h = self._lib.oivf_create(self.d, self.nlist, self.C,
                                        self.n_max, self.n_slabs, self.dir_cap)
        if not self._h:
            raise ValueError("bad oracle parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oivf_destroy(h)
            self._h = None

    # -- mutation --------------------------------------------------------
    def set_centroids(self, c) -> None:
        c = _f32(c)
        assert c.shape == (self.nlist, self.d)
        self._c = c
        self._lib.oivf_set_centroids(self._h, _ptr(c))

    def add(self, ids, x) -> int:
        ids, x = _i64(ids), _f32(x).reshape(-1, self.d)
        assert ids.shape[0] == x.shape[0]
        out = np.zeros(1, np.int64)
        st = self._lib.oivf_add(self._h, _ptr(ids), _ptr(x), ids.shape[0],
                                _ptr(out))
        if st:
            raise OracleError(st)
        return int(out[0])

    def remove(self, ids) -> int:
        ids = _i64(ids)
        out = np.zeros(1, np.int64)
        st = self._lib.oivf_remove(self._h, _ptr(ids), ids.shape[0], _ptr(out))
        if st:
            raise OracleError(st)
        return int(out[0])

    def compact(self, min_free: int = 1, max_moves: int = 1 << 62):
        """Compaction pass: (slabs freed, members rewritten)."""
        fr = np.zeros(1, np.int64)
        mv = np.zeros(1, np.int64)
        st = self._lib.oivf_compact(self._h, int(min_free), int(max_moves), _ptr(fr), _ptr(mv))
        if st:
            raise OracleError(st)
        return int(fr[0]), int(mv[0])

    # -- queries ---------------------------------------------------------
    def assign(self, x) -> np.ndarray:
        x = _f32(x).reshape(-1, self.d)
        out = np.zeros(x.shape[0], np.int32)
        st = self._lib.oivf_assign(self._h, _ptr(x), x.shape[0], _ptr(out))
        if st:
            raise OracleError(st)
        return out

    def probe(self, q, nprobe: int) -> np.ndarray:
        q = _f32(q).reshape(-1, self.d)
        out = np.zeros((q.shape[0], nprobe), np.int32)
        st = self._lib.oivf_probe(self._h, _ptr(q), q.shape[0], nprobe,
                                  _ptr(out))
        if st:
            raise OracleError(st)
        return out

    def search(self, q, k: int, nprobe: int):
        q = _f32(q).reshape(-1, self.d)
        dist = np.zeros((q.shape[0], k), np.float64)
        ids = np.zeros((q.shape[0], k), np.int64)
        st = self._lib.oivf_search(self._h, _ptr(q), q.shape[0], k, nprobe,
                                   _ptr(dist), _ptr(ids))
        if st:
            raise OracleError(st)
        return dist, ids

    def search_with_probes(self, q, k: int, probes):
        q = _f32(q).reshape(-1, self.d)
        probes = np.ascontiguousarray(probes, dtype=np.int32)
        P = probes.shape[1]
        dist = np.zeros((q.shape[0], k), np.float64)
        ids = np.zeros((q.shape[0], k), np.int64)
        st = self._lib.oivf_search_with_probes(self._h, _ptr(q), q.shape[0], k,
                                               P, _ptr(probes), _ptr(dist),
                                               _ptr(ids))
        if st:
            raise OracleError(st)
        return dist, ids

    def exact_knn(self, q, k: int):
        q = _f32(q).reshape(-1, self.d)
        dist = np.zeros((q.shape[0], k), np.float64)
        ids = np.zeros((q.shape[0], k), np.int64)
        st = self._lib.oivf_exact_knn(self._h, _ptr(q), q.shape[0], k,
                                      _ptr(dist), _ptr(ids))
        if st:
            raise OracleError(st)
        return dist, ids

    # -- introspection ---------------------------------------------------
    @property
    def ntotal(self) -> int:
        return int(self._lib.oivf_ntotal(self._h))

    @property
    def free_slabs(self) -> int:
        return int(self._lib.oivf_free_slabs(self._h))

    def list_of(self, id_: int) -> int:
        return int(self._lib.oivf_list_of(self._h, int(id_)))

    def list_size(self, l: int) -> int:
        return int(self._lib.oivf_list_size(self._h, l))

    def list_members(self, l: int):
        """(ids, slab sequence number, slot) of list l in insertion order."""
        n = self.list_size(l)
        ids = np.zeros(n, np.int64)
        seq = np.zeros(n, np.int32)
        slot = np.zeros(n, np.int32)
        self._lib.oivf_list_members(self._h, l, _ptr(ids), _ptr(seq),
                                    _ptr(slot))
        return ids, seq, slot

    def list_vectors(self, l: int) -> np.ndarray:
        x = np.zeros((self.list_size(l), self.d), np.float32)
        self._lib.oivf_list_vectors(self._h, l, _ptr(x))
        return x

    def list_slabs(self, l: int):
        """(fill, live) of the slabs of list l, oldest first."""
        n = int(self._lib.oivf_list_nslabs(self._h, l))
        fill = np.zeros(n, np.int32)
        live = np.zeros(n, np.int32)
        self._lib.oivf_list_slabs(self._h, l, _ptr(fill), _ptr(live))
        return fill, live

    def membership(self) -> np.ndarray:
        """list of every id in [0, n_max), -1 where absent."""
        return np.array([self.list_of(i) for i in range(self.n_max)],
                        dtype=np.int32)


def dists(q, x) -> np.ndarray:
    """FP64 squared distances of one query to each row of x."""
    q = _f32(q).reshape(-1)
    x = _f32(x).reshape(-1, q.shape[0])
    out = np.zeros(x.shape[0], np.float64)
    _load().oivf_dists(_ptr(q), _ptr(x), x.shape[0], q.shape[0], _ptr(out))
    return out


def approx_dists(q, xs, dtype: str, inv_l=None, cent_l=None):
    """FP64 value of the reduced-precision scan's approximate distance of
    one query q to rows xs, and a magnitude for its FP32 accumulation error
    (see ``oivf_approx_dists``).  BF16: ||q||^2 + ||x||^2 - 2 q^.x^ with the
    rounded vectors.  FP8: the residuals from each row's list centroid
    (``cent_l``, one row per member) coded in E4M3, the row's with its
    list's inverse scale (``inv_l``), the query's with 448 / (2 max|q - c|);
    the dot product is scaled back by both.  Returns (dist, mag)."""
    q = _f32(q).reshape(-1)
    xs = _f32(xs).reshape(-1, q.shape[0])
    n, d = xs.shape
    out = np.zeros(n, np.float64)
    mag = np.zeros(n, np.float64)
    if dtype == "bf16":
        _load().oivf_approx_dists(_ptr(q), _ptr(xs), n, d, 0, None, None, _ptr(out), _ptr(mag))
    elif dtype == "fp8":
        cent_l = _f32(cent_l).reshape(n, d)
        inv_l = _f32(inv_l).reshape(n)
        _load().oivf_approx_dists(_ptr(q), _ptr(xs), n, d, 1, _ptr(cent_l), _ptr(inv_l),
                                  _ptr(out), _ptr(mag))
    else:
        raise ValueError(dtype)
    return out, mag


# -- encodings -----------------------------------------------------------
def to_bf16(x) -> np.ndarray:
    x = _f32(x)
    out = np.zeros(x.shape, np.uint16)
    _load().oivf_to_bf16(_ptr(x), _ptr(out), x.size)
    return out


def from_bf16(b) -> np.ndarray:
    b = np.ascontiguousarray(b, dtype=np.uint16)
    out = np.zeros(b.shape, np.float32)
    _load().oivf_from_bf16(_ptr(b), _ptr(out), b.size)
    return out


def to_e4m3(x, inv_scale: float) -> np.ndarray:
    x = _f32(x)
    out = np.zeros(x.shape, np.uint8)
    _load().oivf_to_e4m3(_ptr(x), float(np.float32(inv_scale)), _ptr(out),
                         x.size)
    return out


def from_e4m3(c) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.uint8)
    out = np.zeros(c.shape, np.float64)
    _load().oivf_from_e4m3(_ptr(c), _ptr(out), c.size)
    return out


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 from state `seed` (uint64)."""
    out = np.empty(n, np.uint64)
    _load().oivf_splitmix64(C.c_uint64(seed), n, _ptr(out))
    return out


def kmeans_init_rows(n: int, nlist: int, seed: int) -> np.ndarray:
    """The nlist distinct training rows the k-means starts from."""
    rows = np.empty(nlist, np.int64)
    if _load().oivf_kmeans_init_rows(n, nlist, C.c_uint64(seed), _ptr(rows)):
        raise OracleError(E_ARG)
    return rows


def kmeans(x, nlist: int, iters: int, seed: int):
    """Lloyd's k-means (the reading documented in sivf_oracle.c): returns
    (centroids float32 [nlist, d], final assignment int32 [n])."""
    x = _f32(x)
    n, d = x.shape
    cent = np.empty((nlist, d), np.float32)
    lab = np.empty(n, np.int32)
    st = _load().oivf_kmeans(_ptr(x), n, d, nlist, iters, C.c_uint64(seed), _ptr(cent), _ptr(lab))
    if st:
        raise OracleError(st)
    return cent, lab


def fp8_list_scales(cent) -> np.ndarray:
    """Per-list FP8 inverse scales of the residual codes (see sivf_oracle.c)."""
    cent = _f32(cent)
    out = np.empty(cent.shape[0], np.float32)
    _load().oivf_fp8_list_scales(_ptr(cent), cent.shape[0], cent.shape[1], _ptr(out))
    return out
