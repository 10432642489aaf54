"""ctypes binding of libsivf (include/sivf.h).

The module-level functions carry the C names and only marshal arguments:
torch tensors become device pointers, the torch current stream becomes the
``cudaStream_t``.  Every step of the index runs in the CUDA library; there is
no fallback.  If ``libsivf.so`` has not been built, loading fails loudly.

``Index`` is a small convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsivf.so")

OK, E_ARG, E_NOMEM, E_STATE, E_CUDA, E_CORRUPT, E_TIMEOUT = range(7)
STATUS_NAMES = ["OK", "E_ARG", "E_NOMEM", "E_STATE", "E_CUDA", "E_CORRUPT",
                "E_TIMEOUT"]
FP32, BF16, FP8E4M3 = 0, 1, 2
DTYPES = {"fp32": FP32, "bf16": BF16, "fp8": FP8E4M3, "fp8e4m3": FP8E4M3}

# every symbol include/sivf.h declares
EXPORTS = [
    "sivf_create", "sivf_destroy", "sivf_set_centroids", "sivf_set_list_scales",
    "sivf_train", "sivf_get_centroids", "sivf_assign_stage", "sivf_save", "sivf_load",
    "sivf_reserve", "sivf_add", "sivf_remove", "sivf_compact", "sivf_search",
    "sivf_search_with_probes", "sivf_search_noalloc", "sivf_search_candidates",
    "sivf_assign", "sivf_probe", "sivf_sync",
    "sivf_stats", "sivf_dump", "sivf_dump_payload", "sivf_list_sizes",
    "sivf_profile", "sivf_profile_read", "sivf_last_error", "sivf_version",
    "sivf_set_wait_limit", "sivf_debug_set_error_bits", "sivf_set_chunk_bytes",
    "sivf_set_tile", "sivf_get_tile", "sivf_autotune",
    "sivf_exec_create", "sivf_exec_launch", "sivf_exec_results", "sivf_exec_kernels",
    "sivf_exec_destroy",
    "sivf_server_create", "sivf_server_now_ns", "sivf_server_submit", "sivf_server_wait",
    "sivf_server_drain", "sivf_server_stats", "sivf_server_destroy",
]

OP_ADD, OP_REMOVE, OP_SEARCH, OP_COMPACT = 0, 1, 2, 3


class sivf_config(C.Structure):
    _fields_ = [("d", C.c_int), ("nlist", C.c_int), ("slab_size", C.c_int),
                ("n_max", C.c_int64), ("n_slabs", C.c_int64),
                ("dir_cap", C.c_int64), ("scan_dtypes", C.c_uint32)]


class sivf_stats_t(C.Structure):
    _fields_ = [("ntotal", C.c_int64), ("free_slabs", C.c_int64),
                ("used_slabs", C.c_int64), ("error_bits", C.c_uint32),
                ("last_status", C.c_int32), ("last_count", C.c_int64),
                ("bytes_device", C.c_int64), ("pairs_scanned", C.c_int64),
                ("slab_bytes_scanned", C.c_int64), ("list_bytes_scanned", C.c_int64)]


class sivf_tile(C.Structure):
    _fields_ = [("queries_per_tile", C.c_int32), ("slabs_per_chunk", C.c_int32),
                ("items_per_sm", C.c_int32), ("select_slabs", C.c_int32),
                ("nearest_first", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class sivf_op(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("k", C.c_int32),
                ("nprobe", C.c_int32), ("n", C.c_int64), ("ids", C.c_void_p),
                ("x", C.c_void_p), ("dist", C.c_void_p), ("labels", C.c_void_p)]


class sivf_op_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("pad", C.c_int32), ("count", C.c_int64),
                ("device_ms", C.c_double)]


class sivf_server_config(C.Structure):
    _fields_ = [("k", C.c_int32), ("nprobe", C.c_int32), ("dtype", C.c_int32),
                ("depth", C.c_int32), ("max_query_batch", C.c_int32),
                ("max_insert_batch", C.c_int32), ("max_delete_batch", C.c_int32),
                ("compact_min_free", C.c_int32)]


class sivf_request_info(C.Structure):
    _fields_ = [("kind", C.c_int32), ("status", C.c_int32), ("count", C.c_int64),
                ("batch", C.c_int64), ("latency_ms", C.c_double), ("queue_ms", C.c_double)]


class sivf_server_stats_t(C.Structure):
    _fields_ = [("requests", C.c_int64 * 3), ("batches", C.c_int64 * 3),
                ("items", C.c_int64 * 3), ("deferred", C.c_int64), ("rejected", C.c_int64),
                ("max_in_flight", C.c_int64), ("compact_passes", C.c_int64),
                ("compact_freed", C.c_int64), ("compact_moved", C.c_int64)]


class SivfError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"sivf {name}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libsivf.so and declare its signatures (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing: build it with paper_2601_11808_gb300.build.build()")
        lib = C.CDLL(p)
        vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
        sig = {
            "sivf_create": (i32, [C.POINTER(sivf_config), C.POINTER(vp)]),
            "sivf_destroy": (i32, [vp]),
            "sivf_set_centroids": (i32, [vp, vp, vp]),
            "sivf_train": (i32, [vp, vp, i64, i32, C.c_uint64, vp]),
            "sivf_get_centroids": (i32, [vp, vp, vp]),
            "sivf_assign_stage": (i32, [vp]),
            "sivf_save": (i32, [vp, C.c_char_p, vp]),
            "sivf_load": (i32, [C.c_char_p, C.POINTER(vp)]),
            "sivf_set_list_scales": (i32, [vp, vp, vp]),
            "sivf_reserve": (i32, [vp, i64, i64, i64, i32, i32, vp]),
            "sivf_add": (i32, [vp, vp, vp, i64, vp, C.POINTER(i64)]),
            "sivf_remove": (i32, [vp, vp, i64, vp, C.POINTER(i64)]),
            "sivf_compact": (i32, [vp, i32, i64, vp, C.POINTER(i64), C.POINTER(i64)]),
            "sivf_search": (i32, [vp, vp, i64, i32, i32, i32, vp, vp, vp]),
            "sivf_search_with_probes": (i32, [vp, vp, i64, i32, i32, vp, i32, vp, vp, vp]),
            "sivf_search_noalloc": (i32, [vp, vp, i64, i32, i32, vp, vp, vp]),
            "sivf_search_candidates": (i32, [vp, vp, i64, i32, i32, i32, vp, vp, vp]),
            "sivf_assign": (i32, [vp, vp, i64, vp, vp]),
            "sivf_probe": (i32, [vp, vp, i64, i32, vp, vp]),
            "sivf_sync": (i32, [vp, vp, C.POINTER(i64)]),
            "sivf_stats": (i32, [vp, vp, C.POINTER(sivf_stats_t)]),
            "sivf_dump": (i32, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(i64)]),
            "sivf_dump_payload": (i32, [vp, vp, vp, vp, vp, vp]),
            "sivf_list_sizes": (i32, [vp, vp, vp]),
            "sivf_profile": (i32, [vp, i32]),
            "sivf_set_wait_limit": (i32, [vp, i64]),
            "sivf_set_chunk_bytes": (i32, [vp, i64]),
            "sivf_debug_set_error_bits": (i32, [vp, C.c_uint32, vp]),
            "sivf_profile_read": (i32, [vp, C.c_char_p, C.POINTER(i64), C.POINTER(C.c_double)]),
            "sivf_last_error": (C.c_char_p, [vp]),
            "sivf_set_tile": (i32, [vp, i32, i64, i32, i32, C.POINTER(sivf_tile)]),
            "sivf_get_tile": (i32, [vp, i32, i64, i32, i32, C.POINTER(sivf_tile)]),
            "sivf_autotune": (i32, [vp, vp, i64, i32, i32, i32, i32, vp,
                                    C.POINTER(sivf_tile), C.POINTER(C.c_double)]),
            "sivf_exec_create": (i32, [vp, C.POINTER(sivf_op), i32, C.POINTER(vp)]),
            "sivf_exec_launch": (i32, [vp, vp]),
            "sivf_exec_results": (i32, [vp, vp, C.POINTER(sivf_op_result)]),
            "sivf_exec_kernels": (i64, [vp]),
            "sivf_exec_destroy": (i32, [vp]),
            "sivf_server_create": (i32, [vp, C.POINTER(sivf_server_config), C.POINTER(vp)]),
            "sivf_server_now_ns": (i64, []),
            "sivf_server_submit": (i32, [vp, i32, i64, vp, vp, i64, vp, vp, vp, i64,
                                         C.POINTER(i64)]),
            "sivf_server_wait": (i32, [vp, i64, i64, C.POINTER(sivf_request_info)]),
            "sivf_server_drain": (i32, [vp, i64]),
            "sivf_server_stats": (i32, [vp, C.POINTER(sivf_server_stats_t)]),
            "sivf_server_destroy": (i32, [vp]),
            "sivf_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


# ------------------------------------------------------------ marshalling
def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream=None) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _check(lib, h, st: int):
    if st != OK:
        msg = lib.sivf_last_error(h) if h else b""
        raise SivfError(st, (msg or b"").decode())


def _dev(t, dtype):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor")
    return t


# ------------------------------------------------- C-named entry points
def sivf_version() -> str:
    return load().sivf_version().decode()


def sivf_create(d, nlist, slab_size, n_max, n_slabs, dir_cap=0, scan_dtypes=0) -> int:
    lib = load()
    cfg = sivf_config(int(d), int(nlist), int(slab_size), int(n_max), int(n_slabs),
                      int(dir_cap), int(scan_dtypes))
    h = C.c_void_p()
    _check(lib, None, lib.sivf_create(C.byref(cfg), C.byref(h)))
    return h.value


def sivf_destroy(h) -> None:
    load().sivf_destroy(h)


def sivf_save(h, path: str, stream=None) -> None:
    lib = load()
    _check(lib, h, lib.sivf_save(h, os.fsencode(path), _stream(stream)))


def sivf_load(path: str) -> int:
    lib = load()
    h = C.c_void_p()
    _check(lib, None, lib.sivf_load(os.fsencode(path), C.byref(h)))
    return h.value


def sivf_set_centroids(h, c, stream=None) -> None:
    import torch
    lib = load()
    _check(lib, h, lib.sivf_set_centroids(h, _ptr(_dev(c, torch.float32)), _stream(stream)))


def sivf_train(h, x, iters: int, seed: int, stream=None) -> None:
    import torch
    lib = load()
    xx = _dev(x, torch.float32)
    _check(lib, h, lib.sivf_train(h, _ptr(xx), xx.shape[0], iters, C.c_uint64(seed),
                                  _stream(stream)))


def sivf_get_centroids(h, out, stream=None) -> None:
    import torch
    lib = load()
    _check(lib, h, lib.sivf_get_centroids(h, _ptr(_dev(out, torch.float32)), _stream(stream)))


def sivf_assign_stage(h) -> int:
    return int(load().sivf_assign_stage(h))


def sivf_set_list_scales(h, inv_scale, stream=None) -> None:
    import torch
    lib = load()
    _check(lib, h, lib.sivf_set_list_scales(h, _ptr(_dev(inv_scale, torch.float32)),
                                            _stream(stream)))


def sivf_reserve(h, max_add=0, max_remove=0, max_queries=0, max_k=0, max_nprobe=0,
                 stream=None) -> None:
    lib = load()
    _check(lib, h, lib.sivf_reserve(h, max_add, max_remove, max_queries, max_k,
                                    max_nprobe, _stream(stream)))


def sivf_add(h, ids, x, stream=None, sync=False):
    import torch
    lib = load()
    _dev(ids, torch.int64)
    _dev(x, torch.float32)
    out = C.c_int64(0)
    st = lib.sivf_add(h, _ptr(ids), _ptr(x), ids.numel(), _stream(stream),
                      C.byref(out) if sync else None)
    _check(lib, h, st)
    return out.value if sync else None


def sivf_remove(h, ids, stream=None, sync=False):
    import torch
    lib = load()
    _dev(ids, torch.int64)
    out = C.c_int64(0)
    st = lib.sivf_remove(h, _ptr(ids), ids.numel(), _stream(stream),
                         C.byref(out) if sync else None)
    _check(lib, h, st)
    return out.value if sync else None


def sivf_compact(h, min_free=1, max_moves=1 << 40, stream=None, sync=False):
    """One compaction pass; with sync, (slabs freed, members rewritten)."""
    lib = load()
    fr, mv = C.c_int64(0), C.c_int64(0)
    st = lib.sivf_compact(h, int(min_free), int(max_moves), _stream(stream),
                          C.byref(fr) if sync else None, C.byref(mv) if sync else None)
    _check(lib, h, st)
    return (fr.value, mv.value) if sync else None


def sivf_search(h, q, k, nprobe, dtype=FP32, dist=None, labels=None, stream=None):
    import torch
    lib = load()
    _dev(q, torch.float32)
    nq = q.shape[0]
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.float32, device=q.device)
    if labels is None:
        labels = torch.empty((nq, k), dtype=torch.int64, device=q.device)
    st = lib.sivf_search(h, _ptr(q), nq, k, nprobe, int(dtype), _ptr(dist), _ptr(labels),
                         _stream(stream))
    _check(lib, h, st)
    return dist, labels


def sivf_search_candidates(h, q, kc, nprobe, dtype=BF16, stream=None):
    """The kc best reduced-precision candidates of each query (approximate
    distances and ids), before the FP32 re-rank."""
    import torch
    lib = load()
    _dev(q, torch.float32)
    nq = q.shape[0]
    dist = torch.empty((nq, kc), dtype=torch.float32, device=q.device)
    labels = torch.empty((nq, kc), dtype=torch.int64, device=q.device)
    st = lib.sivf_search_candidates(h, _ptr(q), nq, kc, nprobe, int(dtype), _ptr(dist),
                                    _ptr(labels), _stream(stream))
    _check(lib, h, st)
    return dist, labels


def sivf_search_noalloc(h, q, k, nprobe, dist, labels, stream=None):
    """FP32 search that allocates no device memory during the call: the
    caller passes the output tensors (dist float32 [nq, k], labels int64
    [nq, k]); the library takes its scratch from a fixed device array."""
    import torch
    lib = load()
    _dev(q, torch.float32)
    _dev(dist, torch.float32)
    _dev(labels, torch.int64)
    nq = q.shape[0]
    if tuple(dist.shape) != (nq, k) or tuple(labels.shape) != (nq, k):
        raise ValueError("dist and labels must be [nq, k]")
    st = lib.sivf_search_noalloc(h, _ptr(q), nq, k, nprobe, _ptr(dist), _ptr(labels),
                                 _stream(stream))
    _check(lib, h, st)
    return dist, labels


def sivf_search_with_probes(h, q, k, probes, dtype=FP32, dist=None, labels=None,
                            stream=None):
    import torch
    lib = load()
    _dev(q, torch.float32)
    _dev(probes, torch.int32)
    nq = q.shape[0]
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.float32, device=q.device)
    if labels is None:
        labels = torch.empty((nq, k), dtype=torch.int64, device=q.device)
    st = lib.sivf_search_with_probes(h, _ptr(q), nq, k, probes.shape[1], _ptr(probes),
                                     int(dtype), _ptr(dist), _ptr(labels), _stream(stream))
    _check(lib, h, st)
    return dist, labels


def sivf_assign(h, x, labels=None, stream=None):
    import torch
    lib = load()
    _dev(x, torch.float32)
    if labels is None:
        labels = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
    _check(lib, h, lib.sivf_assign(h, _ptr(x), x.shape[0], _ptr(labels), _stream(stream)))
    return labels


def sivf_probe(h, q, nprobe, probes=None, stream=None):
    import torch
    lib = load()
    _dev(q, torch.float32)
    if probes is None:
        probes = torch.empty((q.shape[0], nprobe), dtype=torch.int32, device=q.device)
    _check(lib, h, lib.sivf_probe(h, _ptr(q), q.shape[0], nprobe, _ptr(probes),
                                  _stream(stream)))
    return probes


def sivf_sync(h, stream=None) -> int:
    """Wait for the stream; raise on a rejected batch, return its count."""
    lib = load()
    out = C.c_int64(0)
    _check(lib, h, lib.sivf_sync(h, _stream(stream), C.byref(out)))
    return out.value


def sivf_stats(h, stream=None) -> dict:
    lib = load()
    s = sivf_stats_t()
    _check(lib, h, lib.sivf_stats(h, _stream(stream), C.byref(s)))
    return {f: getattr(s, f) for f, _ in sivf_stats_t._fields_}


def sivf_dump(h, nlist, n_slabs, slab_size, n_max, dir_cap, stream=None) -> dict:
    lib = load()
    W = slab_size // 32
    out = {
        "list_nslabs": np.zeros(nlist, np.int32),
        "list_head": np.zeros(nlist, np.int32),
        "list_dir": np.zeros((nlist, dir_cap), np.int32),
        "slab_meta": np.zeros((n_slabs, 3), np.int32),
        "slab_bits": np.zeros((n_slabs, W), np.uint32),
        "slab_ids": np.zeros((n_slabs, slab_size), np.int64),
        "att": np.zeros(n_max, np.int64),
        "free_stack": np.zeros(n_slabs, np.int32),
    }
    nfree = C.c_int64(0)
    st = lib.sivf_dump(h, _stream(stream), *[_ptr(out[k]) for k in (
        "list_nslabs", "list_head", "list_dir", "slab_meta", "slab_bits", "slab_ids",
        "att", "free_stack")], C.byref(nfree))
    _check(lib, h, st)
    out["n_free"] = nfree.value
    out["free_stack"] = out["free_stack"][: nfree.value]
    return out


def sivf_dump_payload(h, n_slabs, slab_size, d, nlist, x32=True, bf16=False, fp8=False,
                      stream=None) -> dict:
    lib = load()
    rows = n_slabs * slab_size
    out = {"x32": np.zeros((rows, d), np.float32) if x32 else None,
           "xb16": np.zeros((rows, d), np.uint16) if bf16 else None,
           "x8": np.zeros((rows, d), np.uint8) if fp8 else None,
           "inv_scale": np.zeros(nlist, np.float32)}
    st = lib.sivf_dump_payload(h, _stream(stream), _ptr(out["x32"]), _ptr(out["xb16"]),
                               _ptr(out["x8"]), _ptr(out["inv_scale"]))
    _check(lib, h, st)
    return out


def sivf_list_sizes(h, nlist, stream=None) -> np.ndarray:
    lib = load()
    out = np.zeros(nlist, np.int32)
    _check(lib, h, lib.sivf_list_sizes(h, _stream(stream), _ptr(out)))
    return out


def sivf_set_wait_limit(h, ns: int) -> None:
    lib = load()
    _check(lib, h, lib.sivf_set_wait_limit(h, int(ns)))


def sivf_set_chunk_bytes(h, nbytes: int) -> None:
    lib = load()
    _check(lib, h, lib.sivf_set_chunk_bytes(h, int(nbytes)))


def sivf_debug_set_error_bits(h, bits: int, stream=None) -> None:
    lib = load()
    _check(lib, h, lib.sivf_debug_set_error_bits(h, int(bits), _stream(stream)))


def sivf_profile(h, enable: bool) -> None:
    lib = load()
    _check(lib, h, lib.sivf_profile(h, int(bool(enable))))


def sivf_profile_read(h, kernel: str):
    """(launches, total_ms) of a kernel group recorded since sivf_profile."""
    lib = load()
    n, ms = C.c_int64(0), C.c_double(0.0)
    _check(lib, h, lib.sivf_profile_read(h, kernel.encode(), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def sivf_set_tile(h, dtype, nq, k, nprobe, tile: dict | None) -> None:
    """Install (or with None clear) the scan tile of a batch shape's bucket."""
    lib = load()
    t = None
    if tile is not None:
        t = sivf_tile(**{f: int(tile[f]) for f, _ in sivf_tile._fields_})
    _check(lib, h, lib.sivf_set_tile(h, int(dtype), int(nq), int(k), int(nprobe),
                                     C.byref(t) if t is not None else None))


def sivf_get_tile(h, dtype, nq, k, nprobe) -> dict:
    lib = load()
    t = sivf_tile()
    _check(lib, h, lib.sivf_get_tile(h, int(dtype), int(nq), int(k), int(nprobe), C.byref(t)))
    return t.as_dict()


def sivf_autotune(h, q, k, nprobe, dtype=FP32, reps=5, stream=None):
    """Time searches of q over scan tiles and install the fastest for the
    batch's bucket; returns (tile dict, ms per search)."""
    import torch
    lib = load()
    _dev(q, torch.float32)
    t = sivf_tile()
    ms = C.c_double(0.0)
    _check(lib, h, lib.sivf_autotune(h, _ptr(q), q.shape[0], int(k), int(nprobe), int(dtype),
                                     int(reps), _stream(stream), C.byref(t), C.byref(ms)))
    return t.as_dict(), ms.value


class Exec:
    """A recorded queue of add / remove / search / compact batches (sivf_exec).

    ``ops`` is a list of dicts: {"kind": "add", "ids": t, "x": t},
    {"kind": "remove", "ids": t}, {"kind": "search", "q": t, "k": k,
    "nprobe": p, "dtype": "bf16", "dist": t, "labels": t},
    {"kind": "compact", "min_free": 1, "max_moves": m}.  The tensors are
    device buffers that stay bound to the queue: refill them in place
    between launches.  The wrapper keeps references to them."""

    KINDS = {"add": OP_ADD, "remove": OP_REMOVE, "search": OP_SEARCH, "compact": OP_COMPACT}

    def __init__(self, h, ops: list):
        import torch
        lib = load()
        self.h = h
        self._keep = []
        arr = (sivf_op * len(ops))()
        for i, o in enumerate(ops):
            kind = self.KINDS[o["kind"]]
            e = arr[i]
            e.kind = kind
            if kind == OP_COMPACT:
                e.k = int(o.get("min_free", 1))
                e.n = int(o.get("max_moves", 1 << 30))
            elif kind == OP_SEARCH:
                q = _dev(o["q"], torch.float32)
                e.n = q.shape[0]
                e.x = _ptr(q)
                e.k, e.nprobe = int(o["k"]), int(o["nprobe"])
                e.dtype = DTYPES[o.get("dtype", "fp32")]
                e.dist = _ptr(_dev(o["dist"], torch.float32))
                e.labels = _ptr(_dev(o["labels"], torch.int64))
                self._keep += [q, o["dist"], o["labels"]]
            else:
                ids = _dev(o["ids"], torch.int64)
                e.n = ids.numel()
                e.ids = _ptr(ids)
                self._keep.append(ids)
                if kind == OP_ADD:
                    x = _dev(o["x"], torch.float32)
                    e.x = _ptr(x)
                    self._keep.append(x)
        self.nops = len(ops)
        out = C.c_void_p()
        _check(lib, h, lib.sivf_exec_create(h, arr, len(ops), C.byref(out)))
        self.e = out.value
        self.kernels = lib.sivf_exec_kernels(self.e)

    def launch(self, stream=None) -> None:
        lib = load()
        _check(lib, self.h, lib.sivf_exec_launch(self.e, _stream(stream)))

    def results(self, stream=None) -> list:
        """Per batch: (status, count, device_ms) of the last launch."""
        lib = load()
        res = (sivf_op_result * self.nops)()
        _check(lib, self.h, lib.sivf_exec_results(self.e, _stream(stream), res))
        return [(r.status, r.count, r.device_ms) for r in res]

    def close(self) -> None:
        if getattr(self, "e", None):
            load().sivf_exec_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop over an index (sivf_server): submit requests from host
    numpy arrays, wait for them.  The wrapper keeps each request's arrays
    alive until it has been waited for."""

    KINDS = {"add": OP_ADD, "remove": OP_REMOVE, "search": OP_SEARCH}

    def __init__(self, index, k=10, nprobe=32, dtype="fp32", depth=3, max_query_batch=1024,
                 max_insert_batch=16384, max_delete_batch=16384, compact_min_free=0):
        lib = load()
        self.index = index
        self.h = index.h
        self.k, self.d = int(k), index.d
        cfg = sivf_server_config(self.k, int(nprobe), DTYPES[dtype], int(depth),
                                 int(max_query_batch), int(max_insert_batch),
                                 int(max_delete_batch), int(compact_min_free))
        out = C.c_void_p()
        _check(lib, self.h, lib.sivf_server_create(self.h, C.byref(cfg), C.byref(out)))
        self.s = out.value
        self._keep = {}

    @staticmethod
    def now_ns() -> int:
        return int(load().sivf_server_now_ns())

    def _submit(self, kind, n, ids=None, x=None, evict=None, dist=None, labels=None,
                arrival_ns=0):
        lib = load()
        req = C.c_int64(0)
        ne = 0 if evict is None else len(evict)
        st = lib.sivf_server_submit(self.s, kind, int(n), _ptr(ids), _ptr(x), ne, _ptr(evict),
                                    _ptr(dist), _ptr(labels), int(arrival_ns), C.byref(req))
        _check(lib, self.h, st)
        self._keep[req.value] = (ids, x, evict, dist, labels)
        return req.value

    def add(self, ids, x, evict=None, arrival_ns=0) -> int:
        ids = np.ascontiguousarray(ids, np.int64)
        x = np.ascontiguousarray(x, np.float32).reshape(len(ids), self.d)
        ev = None if evict is None or len(evict) == 0 else np.ascontiguousarray(evict, np.int64)
        return self._submit(OP_ADD, len(ids), ids=ids, x=x, evict=ev, arrival_ns=arrival_ns)

    def remove(self, ids, arrival_ns=0) -> int:
        ids = np.ascontiguousarray(ids, np.int64)
        return self._submit(OP_REMOVE, len(ids), ids=ids, arrival_ns=arrival_ns)

    def search(self, q, arrival_ns=0) -> int:
        q = np.ascontiguousarray(q, np.float32).reshape(-1, self.d)
        dist = np.empty((len(q), self.k), np.float32)
        labels = np.empty((len(q), self.k), np.int64)
        return self._submit(OP_SEARCH, len(q), x=q, dist=dist, labels=labels,
                            arrival_ns=arrival_ns)

    def wait(self, req, timeout_us=-1) -> dict:
        """{kind, status, count, batch, latency_ms, queue_ms[, dist, labels]}."""
        lib = load()
        info = sivf_request_info()
        _check(lib, self.h, lib.sivf_server_wait(self.s, int(req), int(timeout_us),
                                                 C.byref(info)))
        out = {f: getattr(info, f) for f, _ in sivf_request_info._fields_}
        keep = self._keep.pop(req, None)
        if keep is not None and info.kind == OP_SEARCH:
            out["dist"], out["labels"] = keep[3], keep[4]
        return out

    def drain(self, timeout_us=-1) -> None:
        lib = load()
        _check(lib, self.h, lib.sivf_server_drain(self.s, int(timeout_us)))

    def stats(self) -> dict:
        lib = load()
        st = sivf_server_stats_t()
        _check(lib, self.h, lib.sivf_server_stats(self.s, C.byref(st)))
        return {"requests": list(st.requests), "batches": list(st.batches),
                "items": list(st.items), "deferred": st.deferred, "rejected": st.rejected,
                "max_in_flight": st.max_in_flight, "compact_passes": st.compact_passes,
                "compact_freed": st.compact_freed, "compact_moved": st.compact_moved}

    def close(self) -> None:
        if getattr(self, "s", None):
            lib = load()
            st = lib.sivf_server_destroy(self.s)
            self.s = None
            self._keep.clear()
            _check(lib, self.h, st)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- convenience
class Index:
    """Owning wrapper: one device index, calls on the torch current stream."""

    def __init__(self, d, nlist, slab_size=32, n_max=1 << 20, n_slabs=None, dir_cap=0,
                 scan_dtypes=()):
        self.d, self.nlist, self.slab_size = int(d), int(nlist), int(slab_size)
        self.n_max = int(n_max)
        self.n_slabs = int(n_slabs if n_slabs is not None else
                           2 * (self.n_max // self.slab_size + self.nlist))
        mask = 0
        for t in scan_dtypes:
            mask |= 1 << DTYPES[t]
        self.scan_dtypes = tuple(scan_dtypes)
        self.h = sivf_create(self.d, self.nlist, self.slab_size, self.n_max, self.n_slabs,
                             dir_cap, mask)
        self.dir_cap = int(dir_cap) if dir_cap else self.n_slabs

    def close(self):
        if getattr(self, "h", None):
            sivf_destroy(self.h)
            self.h = None

    def save(self, path: str, stream=None):
        """Checkpoint the whole index state to a file."""
        sivf_save(self.h, path, stream)

    @classmethod
    def load(cls, path: str):
        """A new index restored from a file written by save()."""
        import struct
        h = sivf_load(path)
        with open(path, "rb") as f:  # the checkpoint header (configuration)
            hdr = f.read(struct.calcsize("<8sIiiiqqqII"))
        _, _, d, nlist, slab, n_max, n_slabs, dir_cap, dtypes, _ = struct.unpack("<8sIiiiqqqII", hdr)
        self = cls.__new__(cls)
        self.h = h
        self.d, self.nlist, self.slab_size = d, nlist, slab
        self.n_max, self.n_slabs, self.dir_cap = n_max, n_slabs, dir_cap
        self.scan_dtypes = tuple(t for t, v in (("bf16", BF16), ("fp8", FP8E4M3)) if dtypes & (1 << v))
        return self

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_centroids(self, c, stream=None):
        sivf_set_centroids(self.h, c, stream)

    def set_list_scales(self, inv_scale, stream=None):
        sivf_set_list_scales(self.h, inv_scale, stream)

    def train(self, x, iters: int, seed: int = 0, stream=None):
        """Lloyd's k-means on the device rows x; installs the centroids."""
        sivf_train(self.h, x, iters, seed, stream)

    def centroids(self, stream=None):
        """The current centroids as a new [nlist, d] float32 CUDA tensor."""
        import torch
        out = torch.empty((self.nlist, self.d), dtype=torch.float32, device="cuda")
        sivf_get_centroids(self.h, out, stream)
        return out

    def reserve(self, max_add=0, max_remove=0, max_queries=0, max_k=0, max_nprobe=0,
                stream=None):
        sivf_reserve(self.h, max_add, max_remove, max_queries, max_k, max_nprobe, stream)

    def add(self, ids, x, stream=None, sync=False):
        return sivf_add(self.h, ids, x, stream, sync)

    def remove(self, ids, stream=None, sync=False):
        return sivf_remove(self.h, ids, stream, sync)

    def compact(self, min_free=1, max_moves=1 << 40, stream=None, sync=True):
        return sivf_compact(self.h, min_free, max_moves, stream, sync)

    def search(self, q, k, nprobe, dtype="fp32", stream=None, dist=None, labels=None):
        return sivf_search(self.h, q, k, nprobe, DTYPES[dtype], dist, labels, stream)

    def search_candidates(self, q, kc, nprobe, dtype="bf16", stream=None):
        return sivf_search_candidates(self.h, q, kc, nprobe, DTYPES[dtype], stream)

    def search_with_probes(self, q, k, probes, dtype="fp32", stream=None):
        return sivf_search_with_probes(self.h, q, k, probes, DTYPES[dtype], None, None,
                                       stream)

    def assign(self, x, stream=None):
        return sivf_assign(self.h, x, None, stream)

    def probe(self, q, nprobe, stream=None):
        return sivf_probe(self.h, q, nprobe, None, stream)

    def sync(self, stream=None):
        return sivf_sync(self.h, stream)

    def stats(self, stream=None):
        return sivf_stats(self.h, stream)

    def dump(self, stream=None):
        return sivf_dump(self.h, self.nlist, self.n_slabs, self.slab_size, self.n_max,
                         self.dir_cap, stream)

    def list_sizes(self, stream=None):
        return sivf_list_sizes(self.h, self.nlist, stream)

    def profile(self, enable=True):
        sivf_profile(self.h, enable)

    def profile_read(self, kernel):
        return sivf_profile_read(self.h, kernel)

    def set_tile(self, dtype, nq, k, nprobe, tile):
        sivf_set_tile(self.h, DTYPES[dtype], nq, k, nprobe, tile)

    def get_tile(self, dtype, nq, k, nprobe):
        return sivf_get_tile(self.h, DTYPES[dtype], nq, k, nprobe)

    def autotune(self, q, k, nprobe, dtype="fp32", reps=5, stream=None):
        return sivf_autotune(self.h, q, k, nprobe, DTYPES[dtype], reps, stream)

    def executor(self, ops):
        return Exec(self.h, ops)

    def dump_payload(self, bf16=False, fp8=False, stream=None):
        return sivf_dump_payload(self.h, self.n_slabs, self.slab_size, self.d, self.nlist,
                                 True, bf16, fp8, stream)
