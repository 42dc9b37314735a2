"""CPU oracle for exact delta-temporal motif counting - test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA path never does, and the two
share no code: this package wraps ``tm_oracle.c`` (plain C),
which implements Algorithm 1 and Algorithm 2 of arXiv 2204.09236 literally
(single thread, or spread over host threads by ranges of first edges),
the brute-force definitions (Def. 2, Def. 3), and the 36-class layout.

Counter layout (numpy uint64 arrays):
    star[3,2,2,2]  Star[Type, d1, d2, d3]   (Sec. IV-A)
    pair[2,2,2]    Pair[d1, d2, d3]         (Sec. IV-A, case (b))
    tri[3,2,2,2]   Tri[Type, di, dj, dk]    (Sec. IV-B)
Type I/II/III = 0/1/2; direction o = 0, in = 1.

Parity status: every function here is pinned in tests/test_oracle.py (worked
examples printed in Sec. IV-A/IV-B, brute force, closed forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_LIB = _BUILD / "liboracle.so"
_SRC = _HERE / "tm_oracle.c"

_lib = None


def build(force: bool = False) -> Path:
    """Compile tm_oracle.c with the host gcc into oracle/_build/liboracle.so."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o",
                               str(tmp), str(_SRC)])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C signatures on a loaded liboracle."""
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.orc_build.restype = P
    lib.orc_build.argtypes = [i64, P, P, P]
    lib.orc_free.argtypes = [P]
    lib.orc_count.argtypes = [P, i64, P, P, P]
    lib.orc_count_entries.argtypes = [P, i64, P, i64, P, P, P]
    lib.orc_count_centre.argtypes = [P, i64, ctypes.c_int32, P, P, P]
    lib.orc_count_mt.argtypes = [P, i64, ctypes.c_int32, i64, P, P, P]
    lib.orc_num_nodes.restype = i64
    lib.orc_num_nodes.argtypes = [P]
    lib.orc_num_entries.restype = i64
    lib.orc_num_entries.argtypes = [P]
    lib.orc_brute.argtypes = [i64, P, P, P, i64, P, P, P]
    lib.orc_brute_classes.argtypes = [i64, P, P, P, i64, P]
    lib.orc_layout.argtypes = [P]
    lib.orc_merge.argtypes = [P, P, P, P]
    lib.orc_class_cells.argtypes = [ctypes.c_int, P, P, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(str(_LIB)))
    return _lib


def _arrs(src, dst, t):
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    t = np.ascontiguousarray(t, np.int64)
    assert src.shape == dst.shape == t.shape
    return src, dst, t


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cells():
    return (np.zeros((3, 2, 2, 2), np.uint64), np.zeros((2, 2, 2), np.uint64),
            np.zeros((3, 2, 2, 2), np.uint64))


class Graph:
    """S_u lists and E_(v,w) lists built on the host (oracle side)."""

    def __init__(self, src, dst, t):
        self._lib = _load()
        self.src, self.dst, self.t = _arrs(src, dst, t)
        self.m = len(self.src)
        h = self._lib.orc_build(self.m, _ptr(self.src), _ptr(self.dst), _ptr(self.t))
        if not h:
            raise ValueError("oracle: invalid graph (negative id or self-loop) or out of memory")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    @property
    def n(self):
        return int(self._lib.orc_num_nodes(self._h))

    def count(self, delta):
        """All centres: Algorithm 1 and Algorithm 2. Returns (star, pair, tri)."""
        s, p, q = _cells()
        if self._lib.orc_count(self._h, int(delta), _ptr(s), _ptr(p), _ptr(q)) != 0:
            raise ValueError("oracle: delta must be >= 0")
        return s, p, q

    def count_mt(self, delta, threads=None, chunk=4096):
        """As count, on `threads` host threads (default: every core): the
        first edges are cut into chunks of `chunk` S_u positions that threads
        take dynamically (Sec. IV-C's inter- and intra-node split). Returns
        (star, pair, tri), equal to count's."""
        threads = int(threads or os.cpu_count() or 1)
        s, p, q = _cells()
        rc = self._lib.orc_count_mt(self._h, int(delta), threads, int(chunk), _ptr(s), _ptr(p),
                                    _ptr(q))
        if rc != 0:
            raise ValueError(f"oracle count_mt: rc={rc} (bad argument or out of memory)")
        return s, p, q

    def count_entries(self, delta, idx):
        """Algorithm 1/2 bodies for the first edges S[idx] only (sampling)."""
        idx = np.ascontiguousarray(idx, np.int64)
        s, p, q = _cells()
        if self._lib.orc_count_entries(self._h, int(delta), _ptr(idx), len(idx), _ptr(s),
                                       _ptr(p), _ptr(q)) != 0:
            raise ValueError("oracle: bad delta or entry index")
        return s, p, q

    def count_centre(self, delta, u):
        s, p, q = _cells()
        if self._lib.orc_count_centre(self._h, int(delta), int(u), _ptr(s), _ptr(p),
                                      _ptr(q)) != 0:
            raise ValueError("oracle: bad delta or centre")
        return s, p, q


def count(src, dst, t, delta):
    return Graph(src, dst, t).count(delta)


def brute(src, dst, t, delta):
    """Every time-ordered triple with span <= delta, classified by definition."""
    lib = _load()
    src, dst, t = _arrs(src, dst, t)
    s, p, q = _cells()
    rc = lib.orc_brute(len(src), _ptr(src), _ptr(dst), _ptr(t), int(delta), _ptr(s), _ptr(p),
                       _ptr(q))
    if rc != 0:
        raise ValueError(f"oracle brute: rc={rc}")
    return s, p, q


def brute_classes(src, dst, t, delta):
    """36 class counts from each instance's edge pattern (Def. 3)."""
    lib = _load()
    src, dst, t = _arrs(src, dst, t)
    out = np.zeros(36, np.uint64)
    rc = lib.orc_brute_classes(len(src), _ptr(src), _ptr(dst), _ptr(t), int(delta), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle brute_classes: rc={rc}")
    return out.reshape(6, 6)


def layout():
    """6x6 array of edge-pattern codes, out[i][j] = M_(i+1)(j+1)."""
    lib = _load()
    buf = ctypes.create_string_buffer(36 * 16)
    lib.orc_layout(buf)
    raw = buf.raw
    return [[raw[16 * (6 * i + j):16 * (6 * i + j + 1)].split(b"\0")[0].decode()
             for j in range(6)] for i in range(6)]


def merge(star, pair, tri):
    """56 cells -> 36 classes; returns (out[6,6], number of classes whose
    isomorphic cells disagree)."""
    lib = _load()
    s = np.ascontiguousarray(star, np.uint64)
    p = np.ascontiguousarray(pair, np.uint64)
    q = np.ascontiguousarray(tri, np.uint64)
    out = np.zeros(36, np.uint64)
    bad = lib.orc_merge(_ptr(s), _ptr(p), _ptr(q), _ptr(out))
    return out.reshape(6, 6), int(bad)


def class_cells(c):
    """The Star/Pair/Tri cells that class c (0..35) occupies, as 0/1 arrays."""
    lib = _load()
    s, p, q = _cells()
    lib.orc_class_cells(int(c), _ptr(s), _ptr(p), _ptr(q))
    return s, p, q
