"""tm_count_noalloc: the count for callers that cannot allocate memory.

Some callers of this library cannot call cudaMalloc while they count: a
serving thread held to a device-memory budget fixed in advance, a process
whose allocator is sized and locked, or code that must not risk the implicit
synchronisation an allocation can cause. tm_count_noalloc keeps its per-graph
counter cells in a fixed device array inside the library instead. These tests
call it through the C ABI and require exactly the counts of tm_count, on two
calls in a row (the shared array keeps the previous call's contents, so the
second call checks that it is cleared). This file is collected last.
"""
import ctypes
import glob
import os

import numpy as np
import pytest

from paper_2204_09236_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_09236_gb300 import build_ext
    build_ext.build()
    from paper_2204_09236_gb300 import tm as _tm
    torch.cuda.init()
    return _tm


@pytest.fixture(scope="module")
def graphs(tm):
    inputs = [(synth.toy_graph(), 10), (synth.random_small(31, 20, 3000, 200), 25),
              (synth.large(scale=0.001), 86400), (synth.hub(scale=0.001), 3600)]
    gs = [tm.build(s, d, t) for (s, d, t), _ in inputs]
    yield gs, [delta for _, delta in inputs]
    for g in gs:
        g.free()


def test_noalloc_equals_tm_count_on_two_calls(tm, graphs):
    gs, deltas = graphs
    want = np.stack([tm.count(g, d) for g, d in zip(gs, deltas)])
    first = tm.count_noalloc(gs, deltas)
    second = tm.count_noalloc(gs, deltas)
    assert (first == want).all()
    assert (second == want).all()
    # a different order and delta: the cells of the earlier calls must not leak in
    rev = tm.count_noalloc(gs[::-1], [d + 1 for d in deltas[::-1]])
    want_rev = np.stack([tm.count(g, d + 1) for g, d in zip(gs[::-1], deltas[::-1])])
    assert (rev == want_rev).all()


def default_pool_bytes():
    """(reserved, used) bytes of the current device's default memory pool,
    the pool the library's other calls allocate from, read through the CUDA
    runtime that torch ships."""
    libdir = os.path.join(os.path.dirname(torch.__file__), "lib")
    cands = sorted(glob.glob(os.path.join(libdir, "libcudart*.so*"))) + \
        sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    if not cands:
        pytest.skip("no CUDA runtime library to query the memory pool")
    rt = ctypes.CDLL(cands[0])
    dev = ctypes.c_int(0)
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    vals = []
    for attr in (5, 7):  # cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        vals.append(v.value)
    return tuple(vals)


def test_noalloc_leaves_the_memory_pool_unchanged(tm, graphs):
    gs, deltas = graphs
    tm.count_noalloc(gs, deltas)  # the first call looks up the array's address
    torch.cuda.synchronize()
    before = default_pool_bytes()
    out = tm.count_noalloc(gs, deltas)
    torch.cuda.synchronize()
    assert default_pool_bytes() == before
    assert out.shape == (len(gs), 6, 6)


def test_noalloc_rejects_more_graphs_than_its_array_holds(tm, graphs):
    gs, _ = graphs
    k = tm.NOALLOC_MAX_GRAPHS + 1
    with pytest.raises(tm.TmError) as e:
        tm.count_noalloc([gs[0]] * k, [10] * k)
    assert e.value.code == tm.TM_EINVAL
    assert tm.count_noalloc([], []).shape == (0, 6, 6)
