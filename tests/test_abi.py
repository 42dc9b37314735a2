"""The C-ABI library builds, loads and exports every symbol include/tm.h
declares; its host-only calls (layout, class fold) agree with the oracle, and
its memory estimate covers a graph's arrays.
No GPU is needed: nothing here launches a kernel."""
import ctypes
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2204_09236_gb300 import build_ext

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    from paper_2204_09236_gb300 import tm
    return tm


def declared_functions():
    text = (ROOT / "include" / "tm.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tm_build", "tm_count", "tm_free", "tm_count_raw", "tm_count_async",
                 "tm_layout", "tm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIBRARY_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIBRARY_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (tm_\w+)", out))
    assert set(declared_functions()) <= exported


def test_library_is_built_for_sm103a():
    # the build compiles every translation unit for sm_103a only; the kernels'
    # run-time architecture is checked on the GPU (tm_kernel_arch, 103)
    assert build_ext.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_layout_matches_oracle(lib):
    assert lib.tm_layout() == oracle.layout()


def test_class_fold_matches_oracle(lib):
    rng = np.random.default_rng(1)
    for c in range(36):
        # a cell vector that satisfies the isomorphism equalities: random class values
        vals = rng.integers(0, 1000, size=36)
        cells = np.zeros(56, np.uint64)
        for k in range(36):
            s, p, q = oracle.class_cells(k)
            flat = np.concatenate([s.reshape(24), p.reshape(8), q.reshape(24)])
            cells[flat.astype(bool)] = vals[k]
        out, bad = lib.tm_merge(cells)
        assert bad == 0
        want, obad = oracle.merge(cells[:24].reshape(3, 2, 2, 2), cells[24:32].reshape(2, 2, 2),
                                  cells[32:].reshape(3, 2, 2, 2))
        assert obad == 0 and (out == want).all()


def test_class_fold_flags_broken_isomorphism(lib):
    cells = np.zeros(56, np.uint64)
    cells[24] = 5  # Pair[o,o,o] without its mirror Pair[in,in,in]
    cells[40] = 2  # a type-II Tri cell without its type-I / type-III cells
    _, bad = lib.tm_merge(cells)
    assert bad == 2


def test_tri_rotation_identity_matches_oracle_classes():
    """The library fills Tri types I and III from type II with
    Tri[II,i,j,k] = Tri[I,!k,!j,!i] = Tri[III,!i,k,j]; the oracle derives each
    class's cells from the definition. They must name the same cells."""
    for c in range(36):
        s, p, q = oracle.class_cells(c)
        if q.sum() == 0:
            continue
        (i, j, k), = np.argwhere(q[1])
        assert q[0, 1 - k, 1 - j, 1 - i] == 1
        assert q[2, 1 - i, k, j] == 1


def test_estimate_covers_the_resident_arrays(lib):
    """tm_estimate_bytes (host arithmetic, no GPU): a graph's resident estimate
    covers its arrays in the worst case (every edge its own node pair, the
    rank-ordered endpoints kept), both figures grow with the graph, and bad
    sizes are rejected."""
    for m, n in [(0, 0), (1, 2), (1000, 50), (60_000_000, 2_500_000)]:
        resident, scratch = lib.tm_estimate_bytes(m, n)
        slots = 16
        while slots < 2 * m:
            slots *= 2
        arrays = (2 * m * 32          # tt, tn, tc, cin, lk
                  + 4 * (n + 1)       # off
                  + 8 * m             # pos_src, pos_dst
                  + 8 * m             # rank-ordered endpoints
                  + 8 * (m + 1)       # pair list
                  + 16 * slots)       # hash at most half full
        assert resident >= arrays, (m, n)
        assert scratch >= 104 * m
    r0, s0 = lib.tm_estimate_bytes(1000, 50)
    r1, s1 = lib.tm_estimate_bytes(2000, 50)
    r2, _ = lib.tm_estimate_bytes(2000, 5000)
    assert r1 > r0 and s1 > s0 and r2 > r1
    with pytest.raises(lib.TmError):
        lib.tm_estimate_bytes(-1, 5)
