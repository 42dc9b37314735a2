"""Python binding of libtm.so (include/tm.h): argument marshalling only.

Every step of the counting path runs in the library's CUDA kernels. The
binding converts numpy arrays (host memory) or torch tensors (host or CUDA
memory) to raw pointers, passes torch's current CUDA stream where a call takes
a stream, and raises TmError for a negative status. There is no CPU fallback:
if libtm.so has not been built, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libtm.so"

TM_OK, TM_EINVAL, TM_ENOMEM, TM_ECUDA, TM_ETIMEOUT, TM_EBUDGET = 0, -1, -2, -3, -4, -5

if not _LIB_PATH.exists():
    raise ImportError(f"{_LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(str(_LIB_PATH))
_P = ctypes.c_void_p
_i64 = ctypes.c_int64
_lib.tm_build.restype = _P
_lib.tm_build.argtypes = [_P, _P, _P, _i64]
_lib.tm_build_async.restype = _P
_lib.tm_build_async.argtypes = [_P, _P, _P, _i64, _P]
_lib.tm_free.argtypes = [_P]
_lib.tm_free_async.argtypes = [_P, _P]
_lib.tm_count.argtypes = [_P, _i64, _P]
_lib.tm_count_raw.argtypes = [_P, _i64, _P, _P, _P]
_lib.tm_count_async.argtypes = [_P, _i64, _P, _P]
_lib.tm_count_centres.argtypes = [_P, _i64, _P, ctypes.c_int32, _P]
_lib.tm_merge.argtypes = [_P, _P]
_lib.tm_layout.argtypes = [_P]
_lib.tm_fill_tri_types.argtypes = [_P]
_lib.tm_count_shard.argtypes = [_P, _i64, _P, ctypes.c_int32, _P]
_lib.tm_stream_create.restype = _P
_lib.tm_stream_create.argtypes = [_i64]
_lib.tm_stream_append.argtypes = [_P, _P, _P, _P, _i64, _P]
_lib.tm_stream_counts.argtypes = [_P, _P, _P]
_lib.tm_stream_edges.restype = _i64
_lib.tm_stream_edges.argtypes = [_P]
_lib.tm_stream_tail.restype = _i64
_lib.tm_stream_tail.argtypes = [_P]
_lib.tm_stream_free.argtypes = [_P]
_lib.tm_kernel_arch.argtypes = [_P]
_lib.tm_graph_nodes.restype = _i64
_lib.tm_graph_nodes.argtypes = [_P]
_lib.tm_graph_edges.restype = _i64
_lib.tm_graph_edges.argtypes = [_P]
_lib.tm_launch_count.restype = ctypes.c_uint64
_lib.tm_count_noalloc.argtypes = [_P, _P, ctypes.c_int32, _P, _P]
_lib.tm_count_batch.argtypes = [_P, _P, ctypes.c_int32, _P]
_lib.tm_count_select.argtypes = [_P, _i64, ctypes.c_int32, _P]
_lib.tm_count_multi.argtypes = [_P, _P, ctypes.c_int32, _P]
_lib.tm_build_many.restype = _P
_lib.tm_build_many.argtypes = [ctypes.c_int32, _P, _P, _P, _P]
_lib.tm_graph_components.restype = ctypes.c_int32
_lib.tm_graph_components.argtypes = [_P]
_lib.tm_count_many.argtypes = [_P, _P, _P]
_lib.tm_batch_config.argtypes = [_i64, ctypes.c_int32]
_lib.tm_batch_get_config.argtypes = [_P, _P]
_lib.tm_tune_batch.argtypes = [_P, _P, ctypes.c_int32, _P, _P, _P]


class _ReqDesc(ctypes.Structure):
    _fields_ = [("key", ctypes.c_int64), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("m", ctypes.c_int64), ("n_hint", ctypes.c_int64),
                ("delta", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "completed", "failed", "pending", "resident_graphs", "resident_bytes",
        "evictions", "builds", "waves", "edges_counted")] + [
        ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lib.tm_server_create.restype = _P
_lib.tm_server_create.argtypes = [_i64, ctypes.c_int32, ctypes.c_int32]
_lib.tm_server_submit.restype = _i64
_lib.tm_server_submit.argtypes = [_P, ctypes.POINTER(_ReqDesc)]
_lib.tm_server_poll.argtypes = [_P, _i64, _P, ctypes.POINTER(ctypes.c_double)]
_lib.tm_server_wait.argtypes = [_P, _i64, _P, ctypes.POINTER(ctypes.c_double), ctypes.c_double]
_lib.tm_server_stats.argtypes = [_P, ctypes.POINTER(_Stats)]
_lib.tm_server_resident.restype = ctypes.c_int32
_lib.tm_server_resident.argtypes = [_P, _P, ctypes.c_int32]
_lib.tm_server_destroy.argtypes = [_P]
_lib.tm_estimate_bytes.argtypes = [_i64, _i64, _P, _P]
_lib.tm_profile_enable.argtypes = [ctypes.c_int]
_lib.tm_profile_read.argtypes = [_P, _P]
_lib.tm_last_error.restype = ctypes.c_char_p
_lib.tm_last_error.argtypes = [ctypes.POINTER(ctypes.c_int)]

LIBRARY_PATH = str(_LIB_PATH)


class TmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def last_error():
    c = ctypes.c_int(0)
    msg = _lib.tm_last_error(ctypes.byref(c)).decode()
    return c.value, msg


def _check(rc):
    if rc < 0:
        code, msg = last_error()
        raise TmError(rc, msg)
    return rc


def _ptr(x, dtype):
    """Pointer of a contiguous array/tensor of `dtype`; returns (ptr, keepalive)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.uint64}[dtype]
            if x.dtype != tdt:
                raise TypeError(f"expected {tdt}, got {x.dtype}")
            x = x.contiguous()
            return ctypes.c_void_p(x.data_ptr() if x.numel() else None), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return (a.ctypes.data_as(ctypes.c_void_p) if a.size else ctypes.c_void_p(None)), a


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Graph:
    """A graph resident on the current CUDA device (tm_build)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    @property
    def n(self):
        return int(_lib.tm_graph_nodes(self._h))

    @property
    def m(self):
        return int(_lib.tm_graph_edges(self._h))

    def free(self):
        if self._h:
            _lib.tm_free(self._h)
            self._h = None

    def free_async(self, stream=None):
        if self._h:
            _lib.tm_free_async(self._h, _stream_handle(stream))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tm_build(src, dst, t):
    """tm_build: src, dst int32[m], t int64[m] (numpy or torch, host or CUDA)."""
    ps, ks = _ptr(src, np.int32)
    pd, kd = _ptr(dst, np.int32)
    pt, kt = _ptr(t, np.int64)
    m = len(ks)
    if not (len(kd) == m and len(kt) == m):
        raise ValueError("src, dst and t must have the same length")
    h = _lib.tm_build(ps, pd, pt, m)
    if not h:
        code, msg = last_error()
        raise TmError(code, msg)
    return Graph(h)


def tm_build_async(src, dst, t, stream=None):
    ps, ks = _ptr(src, np.int32)
    pd, kd = _ptr(dst, np.int32)
    pt, kt = _ptr(t, np.int64)
    h = _lib.tm_build_async(ps, pd, pt, len(ks), _stream_handle(stream))
    if not h:
        code, msg = last_error()
        raise TmError(code, msg)
    return Graph(h)


def tm_count(g, delta):
    """36 class counts as a (6, 6) uint64 array, out[i, j] = M_(i+1)(j+1)."""
    out = np.zeros(36, np.uint64)
    _check(_lib.tm_count(g.handle, int(delta), out.ctypes.data_as(_P)))
    return out.reshape(6, 6)


def tm_count_raw(g, delta):
    """The paper's counters: star[3,2,2,2], pair[2,2,2], tri[3,2,2,2]."""
    s = np.zeros(24, np.uint64)
    p = np.zeros(8, np.uint64)
    q = np.zeros(24, np.uint64)
    _check(_lib.tm_count_raw(g.handle, int(delta), s.ctypes.data_as(_P), p.ctypes.data_as(_P),
                             q.ctypes.data_as(_P)))
    return s.reshape(3, 2, 2, 2), p.reshape(2, 2, 2), q.reshape(3, 2, 2, 2)


def tm_count_async(g, delta, dev_cells, stream=None):
    """Enqueue the count; dev_cells is a CUDA uint64 tensor of 56 elements."""
    pc, keep = _ptr(dev_cells, np.uint64)
    _check(_lib.tm_count_async(g.handle, int(delta), _stream_handle(stream), pc))
    return keep


def tm_count_centres(g, delta, centres):
    c = np.ascontiguousarray(centres, np.int32)
    cells = np.zeros(56, np.uint64)
    _check(_lib.tm_count_centres(g.handle, int(delta), c.ctypes.data_as(_P), len(c),
                                 cells.ctypes.data_as(_P)))
    return split_cells(cells)


NOALLOC_MAX_GRAPHS = 256


def tm_count_noalloc(graphs, deltas, stream=None):
    """Counts several built graphs without allocating any memory
    (tm_count_noalloc); returns a (k, 6, 6) uint64 array."""
    k = len(graphs)
    hs = (ctypes.c_void_p * max(k, 1))(*[g.handle for g in graphs])
    d = np.ascontiguousarray(deltas, np.int64)
    if len(d) != k:
        raise ValueError("one delta per graph")
    out = np.zeros((max(k, 1), 36), np.uint64)
    _check(_lib.tm_count_noalloc(ctypes.cast(hs, _P), d.ctypes.data_as(_P), k,
                                 _stream_handle(stream), out.ctypes.data_as(_P)))
    return out[:k].reshape(k, 6, 6)


def _handles(graphs):
    return (ctypes.c_void_p * max(len(graphs), 1))(*[g.handle for g in graphs])


def tm_count_batch(graphs, deltas):
    """One persistent launch over all graphs; returns (n, 6, 6) uint64."""
    n = len(graphs)
    d = np.ascontiguousarray(deltas, np.int64)
    if len(d) != n:
        raise ValueError("one delta per graph")
    out = np.zeros((max(n, 1), 36), np.uint64)
    hs = _handles(graphs)
    _check(_lib.tm_count_batch(ctypes.cast(hs, _P), d.ctypes.data_as(_P), n,
                               out.ctypes.data_as(_P)))
    return out[:n].reshape(n, 6, 6)


SELECT_STAR_PAIR, SELECT_TRI = 1, 2


def tm_count_select(g, delta, what):
    """Only the Star/Pair counters (what=1), only the Tri counters (what=2),
    or both (3); returns (star, pair, tri)."""
    cells = np.zeros(56, np.uint64)
    _check(_lib.tm_count_select(g.handle, int(delta), int(what), cells.ctypes.data_as(_P)))
    return split_cells(cells)


def tm_count_multi(g, deltas):
    """One graph, several windows, one batched launch; (k, 6, 6) uint64."""
    d = np.ascontiguousarray(deltas, np.int64)
    out = np.zeros((max(len(d), 1), 36), np.uint64)
    _check(_lib.tm_count_multi(g.handle, d.ctypes.data_as(_P), len(d), out.ctypes.data_as(_P)))
    return out[:len(d)].reshape(len(d), 6, 6)


def tm_build_many(graphs):
    """One device graph whose components are the given (src, dst, t) graphs."""
    k = len(graphs)
    keep, ps, pd, pt, ms = [], [], [], [], []
    for s_, d_, t_ in graphs:
        a, ka = _ptr(s_, np.int32)
        b, kb = _ptr(d_, np.int32)
        c, kc = _ptr(t_, np.int64)
        keep += [ka, kb, kc]
        ps.append(a.value)
        pd.append(b.value)
        pt.append(c.value)
        ms.append(len(ka))
    arr = lambda v: (ctypes.c_void_p * max(k, 1))(*v)
    m = np.ascontiguousarray(ms, np.int64)
    h = _lib.tm_build_many(k, ctypes.cast(arr(ps), _P), ctypes.cast(arr(pd), _P),
                           ctypes.cast(arr(pt), _P), m.ctypes.data_as(_P))
    if not h:
        code, msg = last_error()
        raise TmError(code, msg)
    return Graph(h)


def tm_graph_components(g):
    return int(_lib.tm_graph_components(g.handle))


def tm_count_many(g, deltas):
    k = tm_graph_components(g)
    d = np.ascontiguousarray(deltas, np.int64)
    if len(d) != k:
        raise ValueError(f"one delta per component ({k})")
    out = np.zeros((k, 36), np.uint64)
    _check(_lib.tm_count_many(g.handle, d.ctypes.data_as(_P), out.ctypes.data_as(_P)))
    return out.reshape(k, 6, 6)


def tm_batch_config(item_entries=0, blocks_per_sm=0):
    _check(_lib.tm_batch_config(int(item_entries), int(blocks_per_sm)))


def tm_batch_get_config():
    ie = ctypes.c_int64(0)
    b = ctypes.c_int32(0)
    _check(_lib.tm_batch_get_config(ctypes.byref(ie), ctypes.byref(b)))
    return ie.value, b.value


def tm_tune_batch(g, deltas, reps=3):
    d = np.ascontiguousarray(deltas, np.int64)
    ie = ctypes.c_int64(0)
    b = ctypes.c_int32(0)
    ms = ctypes.c_double(0)
    _check(_lib.tm_tune_batch(g.handle, d.ctypes.data_as(_P), int(reps), ctypes.byref(ie),
                              ctypes.byref(b), ctypes.byref(ms)))
    return ie.value, b.value, ms.value


def tm_estimate_bytes(m, n):
    """(resident bytes, build scratch bytes) of a graph, as the server admits it."""
    r = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _check(_lib.tm_estimate_bytes(int(m), int(n), ctypes.byref(r), ctypes.byref(b)))
    return r.value, b.value


estimate_bytes = tm_estimate_bytes


class Server:
    """tm_server_*: continuous-batching count server with resident graphs."""

    def __init__(self, budget_bytes, workers=2, max_wave=64):
        h = _lib.tm_server_create(int(budget_bytes), int(workers), int(max_wave))
        if not h:
            code, msg = last_error()
            raise TmError(code, msg)
        self._h = h

    def submit(self, key, delta, src=None, dst=None, t=None, n_hint=0):
        d = _ReqDesc(key=int(key), delta=int(delta), n_hint=int(n_hint))
        keep = None
        if src is not None:
            a = np.ascontiguousarray(src, np.int32)
            b = np.ascontiguousarray(dst, np.int32)
            c = np.ascontiguousarray(t, np.int64)
            keep = (a, b, c)
            d.src, d.dst, d.t = a.ctypes.data, b.ctypes.data, c.ctypes.data
            d.m = len(a)
        rid = _lib.tm_server_submit(self._h, ctypes.byref(d))
        del keep  # the server copied the edges
        if rid < 0:
            code, msg = last_error()
            raise TmError(int(rid), msg)
        return int(rid)

    def poll(self, rid):
        out = np.zeros(36, np.uint64)
        lat = ctypes.c_double(0)
        rc = _lib.tm_server_poll(self._h, int(rid), out.ctypes.data_as(_P), ctypes.byref(lat))
        if rc < 0:
            code, msg = last_error()
            raise TmError(rc, msg)
        return rc, out.reshape(6, 6), lat.value

    def wait(self, rid, timeout=120.0):
        out = np.zeros(36, np.uint64)
        lat = ctypes.c_double(0)
        rc = _lib.tm_server_wait(self._h, int(rid), out.ctypes.data_as(_P), ctypes.byref(lat),
                                 float(timeout))
        if rc != 0:
            code, msg = last_error()
            raise TmError(rc, msg)
        return out.reshape(6, 6), lat.value

    def stats(self):
        st = _Stats()
        _check(_lib.tm_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _Stats._fields_}

    def resident(self):
        n = _lib.tm_server_resident(self._h, None, 0)
        keys = np.zeros(max(n, 1), np.int64)
        n = _lib.tm_server_resident(self._h, keys.ctypes.data_as(_P), len(keys))
        return [int(k) for k in keys[:min(n, len(keys))]]

    def close(self):
        if self._h:
            _lib.tm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """Incremental counting of an edge stream for one window (tm_stream_*):
    append time-ordered batches; each returns the raw cells it added."""

    def __init__(self, delta):
        h = _lib.tm_stream_create(int(delta))
        if not h:
            code, msg = last_error()
            raise TmError(code, msg)
        self._h = h

    def append(self, src, dst, t):
        s, keep_s = _ptr(src, np.int32)
        d, keep_d = _ptr(dst, np.int32)
        tt, keep_t = _ptr(t, np.int64)
        added = np.zeros(56, np.uint64)
        _check(_lib.tm_stream_append(self._h, s, d, tt, len(src), added.ctypes.data_as(_P)))
        return added

    def counts(self):
        """(56 raw cells, (6, 6) classes) of everything appended so far."""
        cells = np.zeros(56, np.uint64)
        out = np.zeros(36, np.uint64)
        _check(_lib.tm_stream_counts(self._h, cells.ctypes.data_as(_P), out.ctypes.data_as(_P)))
        return cells, out.reshape(6, 6)

    @property
    def edges(self):
        return int(_lib.tm_stream_edges(self._h))

    @property
    def tail(self):
        return int(_lib.tm_stream_tail(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _lib.tm_stream_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split_cells(cells):
    cells = np.asarray(cells, np.uint64).reshape(56)
    return cells[:24].reshape(3, 2, 2, 2), cells[24:32].reshape(2, 2, 2), cells[32:].reshape(3, 2, 2, 2)


def tm_merge(cells):
    """56 raw cells -> ((6, 6) classes, number of inconsistent classes)."""
    c = np.ascontiguousarray(cells, np.uint64).reshape(56)
    out = np.zeros(36, np.uint64)
    bad = _check(_lib.tm_merge(c.ctypes.data_as(_P), out.ctypes.data_as(_P)))
    return out.reshape(6, 6), bad


def tm_count_shard(g, delta, owner, rank):
    """56 raw cells of the centres u with owner[u] == rank (Tri type II only;
    types I/III zero until tm_fill_tri_types of the sum over the ranks)."""
    o, keep = _ptr(owner, np.int32)
    if len(owner) != g.n:
        raise ValueError("owner must have one entry per node")
    cells = np.zeros(56, np.uint64)
    _check(_lib.tm_count_shard(g.handle, int(delta), o, int(rank), cells.ctypes.data_as(_P)))
    return cells


def tm_fill_tri_types(cells):
    """The 56 cells with their Tri type-I/III cells filled from type II (a
    new uint64 array)."""
    c = np.array(cells, np.uint64).reshape(56)
    _check(_lib.tm_fill_tri_types(c.ctypes.data_as(_P)))
    return c


def tm_kernel_arch():
    """Compute capability the library's kernels run as on the current device
    (103 on a GB300)."""
    a = ctypes.c_int32(0)
    _check(_lib.tm_kernel_arch(ctypes.byref(a)))
    return int(a.value)


def tm_layout():
    buf = ctypes.create_string_buffer(36 * 16)
    _check(_lib.tm_layout(buf))
    raw = buf.raw
    return [[raw[16 * (6 * i + j):16 * (6 * i + j + 1)].split(b"\0")[0].decode()
             for j in range(6)] for i in range(6)]


def tm_launch_count():
    return int(_lib.tm_launch_count())


PHASES = ("validate", "time_sort", "incident", "pairs", "star_pair", "tri")


def tm_profile_enable(on=True):
    _lib.tm_profile_enable(1 if on else 0)


def tm_profile_read():
    """{phase: (device ms summed, timed occurrences)} since the last read."""
    ms = np.zeros(len(PHASES), np.float64)
    calls = np.zeros(len(PHASES), np.uint64)
    _check(_lib.tm_profile_read(ms.ctypes.data_as(_P), calls.ctypes.data_as(_P)))
    return {p: (float(ms[i]), int(calls[i])) for i, p in enumerate(PHASES)}


# short aliases
build = tm_build
build_async = tm_build_async
count = tm_count
count_raw = tm_count_raw
count_async = tm_count_async
count_centres = tm_count_centres
count_noalloc = tm_count_noalloc
count_batch = tm_count_batch
count_select = tm_count_select
count_multi = tm_count_multi
build_many = tm_build_many
count_many = tm_count_many
graph_components = tm_graph_components
batch_config = tm_batch_config
batch_get_config = tm_batch_get_config
tune_batch = tm_tune_batch
merge = tm_merge
fill_tri_types = tm_fill_tri_types
count_shard = tm_count_shard
kernel_arch = tm_kernel_arch
layout = tm_layout
launch_count = tm_launch_count
