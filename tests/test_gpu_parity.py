"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

The bar is bit-exact: every one of the 56 raw cells and the 36 classes must
equal the oracle's on the same seeded inputs. Small cases span many tiles and
ragged tails of the sort and counting kernels; the edge cases cover the empty
graph, single edges, delta = 0, equal timestamps, very long same-pair runs,
extreme timestamps and sparse node ids.
"""
import numpy as np
import pytest

import oracle
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


def gpu_cells(tm, s, d, t, delta, device=True):
    if device:
        g = tm.build(torch.from_numpy(np.ascontiguousarray(s)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(d)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(t)).cuda())
    else:
        g = tm.build(s, d, t)
    try:
        star, pair, tri = tm.count_raw(g, delta)
        out = tm.count(g, delta)
    finally:
        g.free()
    return star, pair, tri, out


def assert_parity(tm, s, d, t, deltas, device=True):
    G = oracle.Graph(s, d, t)
    if device:
        g = tm.build(torch.from_numpy(np.ascontiguousarray(s)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(d)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(t)).cuda())
    else:
        g = tm.build(s, d, t)
    try:
        for delta in deltas:
            S, P, Q = G.count(delta)
            star, pair, tri = tm.count_raw(g, delta)
            assert (star == S).all(), ("star", delta, star.ravel(), S.ravel())
            assert (pair == P).all(), ("pair", delta, pair.ravel(), P.ravel())
            assert (tri == Q).all(), ("tri", delta, tri.ravel(), Q.ravel())
            want, bad = oracle.merge(S, P, Q)
            assert bad == 0
            assert (tm.count(g, delta) == want).all()
    finally:
        g.free()


def test_toy_graph(tm):
    s, d, t = synth.toy_graph()
    assert_parity(tm, s, d, t, [0, 1, 4, 10, 20, 1000])


@pytest.mark.parametrize("seed", range(40))
def test_random_tie_heavy(tm, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    m = int(rng.integers(3, 60))
    tr = int(rng.integers(1, 15))
    s, d, t = synth.random_small(9000 + seed, n, m, tr)
    assert_parity(tm, s, d, t, [0, 1, 3, 7, 100])


@pytest.mark.parametrize("seed", range(4))
def test_multi_tile_random(tm, seed):
    """Several sort tiles (4096 items) with ragged tails and dense ties."""
    s, d, t = synth.random_small(300 + seed, 60, 9000 + 1237 * seed, 4000)
    assert_parity(tm, s, d, t, [0, 5, 40, 300])


def test_tiny_workload_against_definition(tm):
    """The 20,000-edge tiny workload at delta = 3600 s: GPU classes equal the
    brute-force enumeration of the definitions and the oracle's cells."""
    s, d, t = synth.tiny()
    star, pair, tri, out = gpu_cells(tm, s, d, t, 3600)
    assert (out == oracle.brute_classes(s, d, t, 3600)).all()
    assert_parity(tm, s, d, t, [0, 60, 3600, 86400])


@pytest.mark.parametrize("scale", [0.001, 0.004])
def test_large_shape_scaled(tm, scale):
    s, d, t = synth.large(scale=scale)
    assert_parity(tm, s, d, t, [600, 86400])


def test_hub_shape_scaled(tm):
    s, d, t = synth.hub(scale=0.002)
    assert_parity(tm, s, d, t, [600, 3600, 86400])


def test_batch_graphs_scaled(tm):
    graphs, deltas = synth.batch(count=6, scale=0.05)
    for (s, d, t), delta in zip(graphs, deltas):
        assert_parity(tm, s, d, t, [int(delta)])


def test_host_and_device_inputs_agree(tm):
    s, d, t = synth.random_small(11, 40, 3000, 500)
    a = gpu_cells(tm, s, d, t, 30, device=True)
    b = gpu_cells(tm, s, d, t, 30, device=False)
    for x, y in zip(a, b):
        assert (x == y).all()


# ------------------------------------------------------------ edge cases


def test_empty_graph(tm):
    z32 = np.zeros(0, np.int32)
    star, pair, tri, out = gpu_cells(tm, z32, z32, np.zeros(0, np.int64), 10, device=False)
    assert star.sum() == 0 and pair.sum() == 0 and tri.sum() == 0 and out.sum() == 0


@pytest.mark.parametrize("m", [1, 2, 3])
def test_few_edges(tm, m):
    s = np.array([0, 1, 2][:m], np.int32)
    d = np.array([1, 2, 0][:m], np.int32)
    t = np.array([5, 6, 7][:m], np.int64)
    assert_parity(tm, s, d, t, [0, 1, 2, 10])


def test_all_same_timestamp(tm):
    s, d, _ = synth.random_small(5, 7, 50, 1)
    t = np.full(50, 123456789, np.int64)
    assert_parity(tm, s, d, t, [0, 1])


def test_long_same_pair_runs(tm):
    """Long E_(v,w) lists: thousands of edges between a few nodes."""
    rng = np.random.default_rng(3)
    m = 6000
    s = rng.integers(0, 3, size=m).astype(np.int32)
    d = ((s + 1 + rng.integers(0, 2, size=m)) % 3).astype(np.int32)
    t = rng.integers(0, 3000, size=m).astype(np.int64)
    assert_parity(tm, s, d, t, [0, 2, 10])


def test_extreme_timestamps(tm):
    rng = np.random.default_rng(4)
    s, d, _ = synth.random_small(6, 6, 40, 1)
    base = -(2 ** 62)
    t = base + rng.integers(0, 20, size=40).astype(np.int64) * (2 ** 58)
    assert_parity(tm, s, d, t, [0, 2 ** 58, 2 ** 60, 2 ** 63 - 1])


@pytest.mark.parametrize("seed", range(2))
def test_wide_time_span_multi_tile(tm, seed):
    """Timestamps spanning 42 bits over many sort tiles: the 64-bit time keys
    (six passes, the first forming its items from the edge arrays) and the
    20-byte entry payloads. Times are multiples of 2^30, so ties survive."""
    s, d, t = synth.random_small(700 + seed, 80, 20000 + 3001 * seed, 1 << 12)
    t = t * (1 << 30) + (1 << 40)
    assert_parity(tm, s, d, t, [0, 1 << 30, 5 << 30, 60 << 30])


def test_sparse_node_ids(tm):
    s, d, t = synth.random_small(8, 8, 200, 40)
    ids = np.array([0, 17, 4095, 70000, 123457, 999999, 3000000, 5000000], np.int32)
    assert_parity(tm, ids[s], ids[d], t, [0, 3, 9])


def test_delta_huge(tm):
    s, d, t = synth.random_small(9, 6, 60, 1000)
    assert_parity(tm, s, d, t, [2 ** 63 - 1])


# ------------------------------------------------------------ invalid input


def test_rejects_invalid_input(tm):
    with pytest.raises(tm.TmError) as e:
        tm.build(np.array([0, 1], np.int32), np.array([1, 1], np.int32), np.array([1, 2], np.int64))
    assert e.value.code == tm.TM_EINVAL
    with pytest.raises(tm.TmError) as e:
        tm.build(np.array([-1], np.int32), np.array([1], np.int32), np.array([1], np.int64))
    assert e.value.code == tm.TM_EINVAL
    with pytest.raises(tm.TmError) as e:
        tm.build(np.array([0, 1], np.int32), np.array([1, 0], np.int32),
                 np.array([-(2 ** 63), 2 ** 63 - 1], np.int64))
    assert e.value.code == tm.TM_EINVAL
    g = tm.build(np.array([0], np.int32), np.array([1], np.int32), np.array([1], np.int64))
    with pytest.raises(tm.TmError) as e:
        tm.count(g, -1)
    assert e.value.code == tm.TM_EINVAL
    g.free()


def test_async_count_matches_sync(tm):
    s, d, t = synth.random_small(12, 30, 2500, 300)
    g = tm.build(s, d, t)
    cells = torch.zeros(56, dtype=torch.uint64, device="cuda")
    tm.count_async(g, 25, cells)
    torch.cuda.synchronize()
    got = cells.cpu().numpy()
    star, pair, tri = tm.count_raw(g, 25)
    assert (got == np.concatenate([star.ravel(), pair.ravel(), tri.ravel()])).all()
    g.free()


def test_count_centres_matches_oracle_per_centre(tm):
    s, d, t = synth.large(scale=0.002)
    G = oracle.Graph(s, d, t)
    g = tm.build(s, d, t)
    deg = np.bincount(np.concatenate([s, d]))
    order = np.argsort(-deg)
    centres = np.concatenate([order[:3], order[10:13], order[200:203], order[-3:]])
    for u in centres:
        S, P, Q = G.count_centre(86400, int(u))
        star, pair, tri = tm.count_centres(g, 86400, [int(u)])
        assert (star == S).all() and (pair == P).all()
        assert (tri[1] == Q[1]).all()
    g.free()


def test_time_ordered_input(tm):
    """Inputs already in time order (as temporal-graph files come) skip the
    time sort; their counts, ties included, still equal the oracle's on the
    same arrays. Checked against the shuffled order of the same edges too:
    with distinct timestamps the (t, id) order, and so every count, does not
    depend on the input order."""
    s, d, t = synth.tiny()
    o = np.argsort(t, kind="stable")
    s2, d2, t2 = s[o], d[o], t[o]
    assert (np.diff(t2) >= 0).all()
    assert_parity(tm, s2, d2, t2, [0, 60, 3600])
    rng = np.random.default_rng(synth.SEED_BASE + 91)
    m = 5000
    ts = np.sort(rng.choice(10**7, m, replace=False)).astype(np.int64)
    ss = rng.integers(0, 300, m).astype(np.int32)
    dd = ((ss + 1 + rng.integers(0, 299, m)) % 300).astype(np.int32)
    sh = rng.permutation(m)
    for delta in (1000, 100000):
        a = gpu_cells(tm, ss, dd, ts, delta)[3]
        b = gpu_cells(tm, ss[sh], dd[sh], ts[sh], delta)[3]
        assert (a == b).all()


def test_kernels_run_as_sm103(tm):
    """The library's kernels are sm_103a code, as the runtime reports them."""
    assert tm.kernel_arch() == 103
