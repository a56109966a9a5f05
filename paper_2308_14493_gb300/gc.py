"""Thin ctypes binding of the C ABI in include/gc.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  All work
runs in the CUDA library ``libgc.so``; if it is missing or cannot be loaded
the first call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GC_OK, GC_EINVAL, GC_ENOMEM, GC_ECUDA, GC_ETIMEOUT = 0, -1, -2, -3, -4
GRAPHLETS = ("3-path", "3-star", "4-cycle", "tailed-triangle", "diamond", "4-clique")

_lock = threading.Lock()
_lib = None


class GCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class gc_options(ctypes.Structure):
    _fields_ = [("alloc", ctypes.c_void_p), ("free", ctypes.c_void_p), ("ctx", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("region_hops", ctypes.c_int32), ("slack", ctypes.c_float),
                ("device", ctypes.c_int32), ("dense_cluster", ctypes.c_int32), ("chunk_threshold", ctypes.c_int32),
                ("local_max_pairs", ctypes.c_int32), ("serial_count", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class gc_stats(ctypes.Structure):
    _fields_ = [("n_ins_raw", ctypes.c_int64), ("n_del_raw", ctypes.c_int64), ("n_ins", ctypes.c_int64),
                ("n_del", ctypes.c_int64), ("repeats", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("noop_ins", ctypes.c_int64), ("noop_del", ctypes.c_int64), ("region_vertices", ctypes.c_int64),
                ("region_entries", ctypes.c_int64), ("edges_a", ctypes.c_int64), ("edges_b", ctypes.c_int64),
                ("Ca", ctypes.c_int64 * 6), ("Cb", ctypes.c_int64 * 6), ("sums_a", ctypes.c_int64 * 6),
                ("sums_b", ctypes.c_int64 * 6), ("num_edges", ctypes.c_int64), ("ms_device", ctypes.c_float),
                ("ms_wall", ctypes.c_float), ("relayouts", ctypes.c_int32), ("path", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4),
                ("ms_stage", ctypes.c_float * 8), ("work_triangles", ctypes.c_int64),
                ("work_wedges", ctypes.c_int64), ("launches", ctypes.c_int32), ("reserved2", ctypes.c_int32 * 3),
                ("C3a", ctypes.c_int64 * 2), ("C3b", ctypes.c_int64 * 2),
                ("work_wedges_heavy", ctypes.c_int64), ("l2_red_heavy", ctypes.c_int64),
                ("l2_atom_heavy", ctypes.c_int64)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            if name.startswith("reserved"):
                continue
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class gc_tuning(ctypes.Structure):
    _fields_ = [("tri_warp_max", ctypes.c_int32), ("tri_small_max", ctypes.c_int32), ("tri_block_max", ctypes.c_int32),
                ("c4_reg_max", ctypes.c_int32), ("c4_warp_max", ctypes.c_int32), ("c4_block_max", ctypes.c_int32),
                ("c4_cta_max", ctypes.c_int64), ("c4_chunk_min", ctypes.c_int64), ("c4_chunk_max", ctypes.c_int64),
                ("local_max_pairs", ctypes.c_int64), ("local_c4_heavy_min", ctypes.c_int64),
                ("pair_min_share", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if not name.startswith("reserved")}


class gc_server_options(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 6)]


class gc_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("graph", ctypes.c_int32), ("status", ctypes.c_int32),
                ("counts", ctypes.c_uint64 * 6), ("n_ins", ctypes.c_int64), ("n_del", ctypes.c_int64),
                ("region_vertices", ctypes.c_int64), ("ms_device", ctypes.c_float), ("relayouts", ctypes.c_int32),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("bytes_predicted", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["counts"] = [int(x) for x in self.counts]
        return d


def library_path() -> str:
    return _build.LIB


def load():
    """Load libgc.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32p = ctypes.POINTER(ctypes.c_int32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.gc_default_options.argtypes = [ctypes.POINTER(gc_options)]
            lib.gc_default_options.restype = None
            lib.gc_open.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.POINTER(gc_options), ctypes.POINTER(P)]
            lib.gc_count_static.argtypes = [P, u64p]
            lib.gc_counts.argtypes = [P, u64p]
            lib.gc_counts3.argtypes = [P, u64p]
            lib.gc_counts_all.argtypes = [P, u64p]
            lib.gc_vertex_counts.argtypes = [P, u64p]
            lib.gc_vertex_orbits.argtypes = [P, u64p]
            lib.gc_edge_counts.argtypes = [P, i32p, u64p]
            lib.gc_edge_orbits.argtypes = [P, i32p, u64p]
            lib.gc_delete_vertices.argtypes = [P, i32p, ctypes.c_int64, u64p]
            lib.gc_add_vertices.argtypes = [P, ctypes.c_int64, i32p]
            lib.gc_num_vertices.argtypes = [P]
            lib.gc_num_vertices.restype = ctypes.c_int32
            lib.gc_apply_batch.argtypes = [P, i32p, ctypes.c_int64, i32p, ctypes.c_int64, u64p]
            lib.gc_apply_batch_device.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int64, u64p]
            lib.gc_count_batch.argtypes = [P, i32p, ctypes.c_int64, i32p, ctypes.c_int64, u64p]
            lib.gc_count_batch_device.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int64, u64p]
            lib.gc_apply_batches.argtypes = [P, ctypes.POINTER(i32p), i64p, ctypes.POINTER(i32p), i64p,
                                             ctypes.c_int32, ctypes.c_int32, u64p]
            lib.gc_apply_batches_device.argtypes = [P, P, i64p, ctypes.c_int32, ctypes.c_int32, u64p]
            lib.gc_batch_stats.argtypes = [P, ctypes.POINTER(gc_stats)]
            lib.gc_num_edges.argtypes = [P]
            lib.gc_num_edges.restype = ctypes.c_int64
            lib.gc_export_csr.argtypes = [P, i32p, i32p]
            lib.gc_last_error.argtypes = [P]
            lib.gc_last_error.restype = ctypes.c_char_p
            lib.gc_close.argtypes = [P]
            lib.gc_close.restype = None
            lib.gc_count_static_noalloc.argtypes = [ctypes.c_int32, P, P, ctypes.c_int64, P, u64p]
            lib.gc_get_tuning.argtypes = [P, ctypes.POINTER(gc_tuning)]
            lib.gc_set_tuning.argtypes = [P, ctypes.POINTER(gc_tuning)]
            lib.gc_autotune.argtypes = [P, ctypes.c_int32, ctypes.POINTER(gc_tuning), ctypes.POINTER(ctypes.c_float)]
            lib.gc_device_bytes.argtypes = [P]
            lib.gc_device_bytes.restype = ctypes.c_int64
            lib.gc_batch_bytes.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
            lib.gc_batch_bytes.restype = ctypes.c_int64
            lib.gc_trim.argtypes = [P]
            lib.gc_server_open.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.POINTER(gc_server_options),
                                           ctypes.POINTER(P)]
            lib.gc_server_submit.argtypes = [P, ctypes.c_int32, i32p, ctypes.c_int64, i32p, ctypes.c_int64, i64p]
            lib.gc_server_wait.argtypes = [P, ctypes.c_int64, ctypes.POINTER(gc_result)]
            lib.gc_server_drain.argtypes = [P]
            lib.gc_server_counters.argtypes = [P, i64p, i64p]
            lib.gc_server_close.argtypes = [P]
            lib.gc_server_close.restype = None
            _lib = lib
    return _lib


def _check(rc: int, h=None):
    if rc != GC_OK:
        msg = load().gc_last_error(h)
        raise GCError(rc, (msg or b"").decode() or "gc call failed")


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, ct=ctypes.c_int32):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _pairs(p):
    a = _i32(np.asarray(p, dtype=np.int32).reshape(-1, 2)) if p is not None else np.zeros((0, 2), np.int32)
    return a, a.shape[0]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator, through
    the gc_options alloc / free callbacks: every buffer the library takes is
    a block of torch's pool, allocated and released in the order of the
    library's stream (the stream the callback receives).  ``live`` maps each
    outstanding pointer to its size; ``fail`` set True (or ``fail_after``
    set to a count of allocations) makes every later allocation return NULL,
    as an exhausted pool would (the library then reports GC_ENOMEM).  Keep
    the object alive while any handle opened with it is open."""

    def __init__(self, device: int | None = None):
        import torch

        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.live: dict[int, int] = {}
        self.allocs = 0
        self.fail = False
        self.fail_after: int | None = None
        self._lock = threading.Lock()
        self._alloc_cb = ALLOC_FN(self._alloc)
        self._free_cb = FREE_FN(self._free)

    def _alloc(self, size, stream, ctx):
        if self.fail or (self.fail_after is not None and self.allocs >= self.fail_after):
            return None
        try:
            p = self._torch.cuda.caching_allocator_alloc(int(size), self.device, int(stream or 0))
        except Exception:  # out of memory: the library sees NULL and returns GC_ENOMEM
            return None
        with self._lock:
            self.live[int(p)] = int(size)
            self.allocs += 1
        return p

    def _free(self, ptr, stream, ctx):
        if not ptr:
            return
        with self._lock:
            self.live.pop(int(ptr), None)
        self._torch.cuda.caching_allocator_delete(int(ptr))

    def options(self, opt) -> None:
        opt.alloc = ctypes.cast(self._alloc_cb, ctypes.c_void_p)
        opt.free = ctypes.cast(self._free_cb, ctypes.c_void_p)
        opt.ctx = None


def gc_open(n: int, row_ptr, col, region_hops: int = 3, slack: float = 0.25, stream: int = 0,
            chunk_threshold: int = 0, dense_cluster: int = 0, local_max_pairs: int = 0,
            allocator: TorchAllocator | None = None, serial_count: bool = False):
    """Open a graph from a symmetric CSR; returns an opaque handle.  With an
    ``allocator`` (e.g. TorchAllocator) the library takes its device memory
    through it instead of cudaMallocAsync."""
    lib = load()
    rp = _i32(row_ptr)
    c = _i32(col) if len(col) else np.zeros(1, np.int32)
    opt = gc_options()
    lib.gc_default_options(ctypes.byref(opt))
    opt.region_hops = region_hops
    opt.slack = slack
    opt.stream = stream or None
    opt.chunk_threshold = chunk_threshold
    opt.dense_cluster = dense_cluster
    opt.local_max_pairs = local_max_pairs
    opt.serial_count = 1 if serial_count else 0
    if allocator is not None:
        allocator.options(opt)
    h = ctypes.c_void_p()
    rc = lib.gc_open(int(n), _ptr(rp), _ptr(c), ctypes.byref(opt), ctypes.byref(h))
    _check(rc, None)
    return h


def gc_close(h) -> None:
    load().gc_close(h)


def gc_count_static(h) -> list[int]:
    out = np.zeros(6, np.uint64)
    _check(load().gc_count_static(h, _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_counts(h) -> list[int]:
    out = np.zeros(6, np.uint64)
    _check(load().gc_counts(h, _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


ALL_TYPES = GRAPHLETS + ("triangle+isolated", "2-path+isolated", "two-disjoint-edges", "edge+2-isolated", "empty")


def gc_counts_all(h) -> list[int]:
    """Induced counts of all eleven 4-vertex graphs (Python ints; 128-bit)."""
    out = np.zeros(22, np.uint64)
    _check(load().gc_counts_all(h, _ptr(out, ctypes.c_uint64)), h)
    return [int(out[2 * i]) | (int(out[2 * i + 1]) << 64) for i in range(11)]


def gc_vertex_counts(h, n: int) -> np.ndarray:
    """Per-vertex graphlet counts of the current graph: uint64[n, 6]."""
    out = np.zeros((max(n, 1), 6), np.uint64)
    _check(load().gc_vertex_counts(h, _ptr(out, ctypes.c_uint64)), h)
    return out[:n]


def gc_vertex_orbits(h, n: int) -> np.ndarray:
    """Per-vertex orbit counts (orbits 4..14) of the current graph: uint64[n, 11]."""
    out = np.zeros((max(n, 1), 11), np.uint64)
    _check(load().gc_vertex_orbits(h, _ptr(out, ctypes.c_uint64)), h)
    return out[:n]


def _edge_rows(h, fn, k: int):
    m = gc_num_edges(h)
    edges = np.zeros((max(m, 1), 2), np.int32)
    out = np.zeros((max(m, 1), k), np.uint64)
    _check(fn(h, _ptr(edges, ctypes.c_int32), _ptr(out, ctypes.c_uint64)), h)
    return edges[:m], out[:m]


def gc_edge_counts(h):
    """Per-edge graphlet counts of the current graph: (int32[m, 2] edges
    lo < hi in increasing order, uint64[m, 6])."""
    return _edge_rows(h, load().gc_edge_counts, 6)


def gc_edge_orbits(h):
    """Per-edge orbit counts (edge orbits 0..9) of the current graph:
    (int32[m, 2] edges, uint64[m, 10])."""
    return _edge_rows(h, load().gc_edge_orbits, 10)


def gc_counts3(h) -> list[int]:
    """Maintained 3-vertex counts: [induced 2-paths, triangles]."""
    out = np.zeros(2, np.uint64)
    _check(load().gc_counts3(h, _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_delete_vertices(h, ids) -> list[int]:
    """Delete every edge of the given vertices (one batch); counts after."""
    a = _i32(np.asarray(ids, dtype=np.int32).reshape(-1)) if ids is not None else np.zeros(0, np.int32)
    buf = a if a.size else np.zeros(1, np.int32)
    out = np.zeros(6, np.uint64)
    _check(load().gc_delete_vertices(h, _ptr(buf), a.size, _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_add_vertices(h, k: int) -> int:
    """Append k isolated vertices; returns the first new id."""
    first = ctypes.c_int32()
    _check(load().gc_add_vertices(h, int(k), ctypes.byref(first)), h)
    return int(first.value)


def gc_num_vertices(h) -> int:
    return int(load().gc_num_vertices(h))


def gc_apply_batch(h, ins, dels) -> list[int]:
    a, na = _pairs(ins)
    d, nd = _pairs(dels)
    out = np.zeros(6, np.uint64)
    _check(load().gc_apply_batch(h, _ptr(a), na, _ptr(d), nd, _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_apply_batch_device(h, d_ins_ptr: int, n_ins: int, d_del_ptr: int, n_del: int) -> list[int]:
    """Pairs already in device memory (raw pointers, e.g. ``tensor.data_ptr()``)."""
    out = np.zeros(6, np.uint64)
    _check(load().gc_apply_batch_device(h, ctypes.c_void_p(d_ins_ptr), n_ins, ctypes.c_void_p(d_del_ptr), n_del,
                                        _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_count_batch(h, ins, dels) -> list[int]:
    """Counts of G (+) B without applying the batch (what-if)."""
    a, na = _pairs(ins)
    d, nd = _pairs(dels)
    out = np.zeros(6, np.uint64)
    _check(load().gc_count_batch(h, _ptr(a), na, _ptr(d), nd, _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_count_batch_device(h, d_ins_ptr: int, n_ins: int, d_del_ptr: int, n_del: int) -> list[int]:
    out = np.zeros(6, np.uint64)
    _check(load().gc_count_batch_device(h, ctypes.c_void_p(d_ins_ptr), n_ins, ctypes.c_void_p(d_del_ptr), n_del,
                                        _ptr(out, ctypes.c_uint64)), h)
    return [int(x) for x in out]


def gc_apply_batches(h, batches, independent: bool = False) -> list[list[int]]:
    k = len(batches)
    arrs = [(_pairs(i), _pairs(d)) for i, d in batches]
    i32p = ctypes.POINTER(ctypes.c_int32)
    ins_p = (i32p * max(k, 1))(*[_ptr(a[0][0]) for a in arrs])
    del_p = (i32p * max(k, 1))(*[_ptr(a[1][0]) for a in arrs])
    n_ins = np.array([a[0][1] for a in arrs] or [0], dtype=np.int64)
    n_del = np.array([a[1][1] for a in arrs] or [0], dtype=np.int64)
    out = np.zeros((max(k, 1), 6), np.uint64)
    _check(load().gc_apply_batches(h, ins_p, _ptr(n_ins, ctypes.c_int64), del_p, _ptr(n_del, ctypes.c_int64), k,
                                   1 if independent else 0, _ptr(out, ctypes.c_uint64)), h)
    return [[int(x) for x in row] for row in out[:k]]


def gc_apply_batches_device(h, d_pairs_ptr: int, batches, independent: bool = False) -> list[list[int]]:
    """Batches whose pairs are in device memory: ``batches`` is a [k][4] array of
    (ins_off, n_ins, del_off, n_del) in pairs relative to ``d_pairs_ptr``."""
    b = np.ascontiguousarray(np.asarray(batches, dtype=np.int64).reshape(-1, 4))
    k = b.shape[0]
    out = np.zeros((max(k, 1), 6), np.uint64)
    _check(load().gc_apply_batches_device(h, ctypes.c_void_p(d_pairs_ptr), _ptr(b, ctypes.c_int64), k,
                                          1 if independent else 0, _ptr(out, ctypes.c_uint64)), h)
    return [[int(x) for x in row] for row in out[:k]]


def gc_batch_stats(h) -> dict:
    s = gc_stats()
    _check(load().gc_batch_stats(h, ctypes.byref(s)), h)
    return s.as_dict()


def gc_num_edges(h) -> int:
    return int(load().gc_num_edges(h))


def gc_export_csr(h, n: int):
    m = gc_num_edges(h)
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(max(2 * m, 1), np.int32)
    _check(load().gc_export_csr(h, _ptr(rp), _ptr(col)), h)
    return rp, col[: 2 * m]


GC_NOALLOC_MAX_VERTICES = 16384
GC_NOALLOC_MAX_ENTRIES = 524288


def gc_count_static_noalloc(n: int, d_row_ptr: int, d_col: int, nnz: int, stream: int = 0) -> list[int]:
    """Static count without any device allocation, for callers that must not
    allocate (memory reserved up front by another allocator, latency-critical
    loops, hosts that forbid allocations after start-up).  The CSR is already
    in device memory: raw pointers (e.g. ``tensor.data_ptr()``) to int32
    row offsets and sorted, symmetric rows.  Limited to
    GC_NOALLOC_MAX_VERTICES vertices and GC_NOALLOC_MAX_ENTRIES entries."""
    out = np.zeros(6, np.uint64)
    rc = load().gc_count_static_noalloc(int(n), ctypes.c_void_p(d_row_ptr), ctypes.c_void_p(d_col), int(nnz),
                                        ctypes.c_void_p(stream or None), _ptr(out, ctypes.c_uint64))
    if rc != GC_OK:
        raise GCError(rc, "gc_count_static_noalloc failed (sizes beyond the fixed scratch, "
                          "a CSR that is not symmetric, simple and sorted, or a CUDA error)")
    return [int(x) for x in out]


def gc_get_tuning(h) -> dict:
    t = gc_tuning()
    _check(load().gc_get_tuning(h, ctypes.byref(t)), h)
    return t.as_dict()


def gc_set_tuning(h, **bounds) -> None:
    t = gc_tuning()
    _check(load().gc_get_tuning(h, ctypes.byref(t)), h)
    for k, v in bounds.items():
        setattr(t, k, int(v))
    _check(load().gc_set_tuning(h, ctypes.byref(t)), h)


def gc_autotune(h, reps: int = 2) -> tuple[dict, float]:
    t = gc_tuning()
    ms = ctypes.c_float()
    _check(load().gc_autotune(h, int(reps), ctypes.byref(t), ctypes.byref(ms)), h)
    return t.as_dict(), float(ms.value)


def gc_device_bytes(h) -> int:
    return int(load().gc_device_bytes(h))


def gc_batch_bytes(h, n_ins: int, n_del: int) -> int:
    return int(load().gc_batch_bytes(h, int(n_ins), int(n_del)))


def gc_trim(h) -> None:
    _check(load().gc_trim(h), h)


def gc_server_open(handles, slots: int = 4, hbm_budget_bytes: int = 0):
    lib = load()
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    o = gc_server_options()
    o.slots = slots
    o.hbm_budget_bytes = hbm_budget_bytes
    s = ctypes.c_void_p()
    rc = lib.gc_server_open(arr, len(handles), ctypes.byref(o), ctypes.byref(s))
    if rc != GC_OK:
        raise GCError(rc, "gc_server_open failed")
    return s


def gc_server_submit(s, graph: int, ins, dels) -> int:
    a, na = _pairs(ins)
    d, nd = _pairs(dels)
    t = ctypes.c_int64()
    rc = load().gc_server_submit(s, int(graph), _ptr(a), na, _ptr(d), nd, ctypes.byref(t))
    if rc != GC_OK:
        raise GCError(rc, "gc_server_submit failed")
    return int(t.value)


def gc_server_wait(s, ticket: int) -> dict:
    r = gc_result()
    rc = load().gc_server_wait(s, int(ticket), ctypes.byref(r))
    if rc != GC_OK:
        raise GCError(rc, "gc_server_wait: unknown ticket")
    return r.as_dict()


def gc_server_drain(s) -> None:
    load().gc_server_drain(s)


def gc_server_counters(s) -> tuple[int, int]:
    a, b = ctypes.c_int64(), ctypes.c_int64()
    load().gc_server_counters(s, ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


def gc_server_close(s) -> None:
    load().gc_server_close(s)


class Server:
    """Request loop over resident graphs (``Graph`` objects, not owned)."""

    def __init__(self, graphs, slots: int = 4, hbm_budget_bytes: int = 0):
        self.graphs = list(graphs)
        self.s = gc_server_open([g.h for g in self.graphs], slots, hbm_budget_bytes)

    def submit(self, graph: int, ins, dels) -> int:
        return gc_server_submit(self.s, graph, ins, dels)

    def wait(self, ticket: int) -> dict:
        return gc_server_wait(self.s, ticket)

    def drain(self):
        gc_server_drain(self.s)

    def counters(self):
        return gc_server_counters(self.s)

    def close(self):
        if self.s is not None:
            gc_server_close(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gc_last_error(h=None) -> str:
    return (load().gc_last_error(h) or b"").decode()


class Graph:
    """A device-resident graph with maintained graphlet counts.

    Each method calls the C entry point of the same name (``counts`` ->
    ``gc_counts``, ``apply`` -> ``gc_apply_batch``, ``apply_many`` ->
    ``gc_apply_batches``, ``edge_orbits`` -> ``gc_edge_orbits``, ...) on the
    handle; ``with Graph(...) as g`` closes it at the end.  The local
    counts (``vertex_*``, ``edge_*``) describe the current graph and leave
    the maintained counts untouched."""

    def __init__(self, n: int, row_ptr, col, region_hops: int = 3, slack: float = 0.25, **opts):
        self.n = int(n)
        self.allocator = opts.get("allocator")  # kept alive as long as the handle
        self.h = gc_open(n, row_ptr, col, region_hops, slack, **opts)

    def close(self):
        if self.h is not None:
            gc_close(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counts(self):
        return gc_counts(self.h)

    def counts3(self):
        return gc_counts3(self.h)

    def counts_all(self):
        return gc_counts_all(self.h)

    def vertex_counts(self):
        return gc_vertex_counts(self.h, self.n)

    def vertex_orbits(self):
        return gc_vertex_orbits(self.h, self.n)

    def edge_counts(self):
        return gc_edge_counts(self.h)

    def edge_orbits(self):
        return gc_edge_orbits(self.h)

    def count_static(self):
        return gc_count_static(self.h)

    def apply(self, ins, dels):
        return gc_apply_batch(self.h, ins, dels)

    def count_batch(self, ins, dels):
        return gc_count_batch(self.h, ins, dels)

    def delete_vertices(self, ids):
        return gc_delete_vertices(self.h, ids)

    def add_vertices(self, k: int) -> int:
        first = gc_add_vertices(self.h, k)
        self.n = gc_num_vertices(self.h)
        return first

    def apply_many(self, batches, independent=False):
        return gc_apply_batches(self.h, batches, independent)

    def stats(self):
        return gc_batch_stats(self.h)

    def num_edges(self):
        return gc_num_edges(self.h)

    def export_csr(self):
        return gc_export_csr(self.h, self.n)

    def device_bytes(self):
        return gc_device_bytes(self.h)

    def tuning(self):
        return gc_get_tuning(self.h)

    def set_tuning(self, **bounds):
        gc_set_tuning(self.h, **bounds)

    def autotune(self, reps: int = 2):
        return gc_autotune(self.h, reps)

    def trim(self):
        gc_trim(self.h)
