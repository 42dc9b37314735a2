"""Batched counting (one persistent launch over many graphs, each with its own
delta) against the oracle and against one-graph-per-launch counting."""
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
    return _tm


def batch_inputs(count=12, scale=0.02):
    graphs, deltas = synth.batch(count=count, scale=scale)
    graphs = list(graphs) + [synth.toy_graph(), synth.random_small(5, 6, 40, 8),
                             (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))]
    deltas = list(int(d) for d in deltas) + [10, 3, 100]
    return graphs, deltas


def oracle_classes(s, d, t, delta):
    if len(s) == 0:
        return np.zeros((6, 6), np.uint64)
    out, bad = oracle.merge(*oracle.count(s, d, t, delta))
    assert bad == 0
    return out


def test_count_batch_equals_oracle_and_single(tm):
    graphs, deltas = batch_inputs()
    gs = [tm.build(*g) for g in graphs]
    got = tm.count_batch(gs, deltas)
    for i, ((s, d, t), delta) in enumerate(zip(graphs, deltas)):
        assert (got[i] == oracle_classes(s, d, t, delta)).all(), i
        assert (got[i] == tm.count(gs[i], delta)).all(), i
    again = tm.count_batch(gs[::-1], deltas[::-1])  # replay with new queue contents
    assert (again == got[::-1]).all()
    for g in gs:
        g.free()


def test_build_many_count_many(tm):
    graphs, deltas = batch_inputs(count=10, scale=0.03)
    g = tm.build_many(graphs)
    assert tm.graph_components(g) == len(graphs)
    got = tm.count_many(g, deltas)
    for i, ((s, d, t), delta) in enumerate(zip(graphs, deltas)):
        assert (got[i] == oracle_classes(s, d, t, delta)).all(), i
    # one window for all: the union count is the sum of the components' counts
    same = tm.count_many(g, [3600] * len(graphs))
    assert (tm.count(g, 3600) == same.sum(axis=0)).all()
    g.free()


def test_item_size_and_grid_do_not_change_counts(tm):
    graphs, deltas = batch_inputs(count=6, scale=0.05)
    g = tm.build_many(graphs)
    base = tm.count_many(g, deltas)
    saved = tm.batch_get_config()
    try:
        for ie, bps in [(256, 1), (1000, 2), (1 << 20, 0)]:
            tm.batch_config(ie, bps)
            assert (tm.count_many(g, deltas) == base).all(), (ie, bps)
        ie, bps, ms = tm.tune_batch(g, deltas, reps=1)
        assert ie >= 256 and ms > 0
        assert (tm.count_many(g, deltas) == base).all()
    finally:
        tm.batch_config(*saved)
    g.free()


def test_build_many_rejects_bad_component(tm):
    ok = synth.toy_graph()
    bad = (np.array([0, 1], np.int32), np.array([1, 1], np.int32), np.array([1, 2], np.int64))
    with pytest.raises(tm.TmError) as e:
        tm.build_many([ok, bad])
    assert e.value.code == tm.TM_EINVAL


def test_count_select_and_multi(tm):
    s, d, t = synth.hub(scale=0.001)
    g = tm.build(s, d, t)
    # the oracle's counters (Algorithm 1: Star and Pair; Algorithm 2: Tri)
    S, P, Q = oracle.count(s, d, t, 3600)
    s1, p1, q1 = tm.count_select(g, 3600, tm.SELECT_STAR_PAIR)
    assert (s1 == S).all() and (p1 == P).all() and q1.sum() == 0
    s2, p2, q2 = tm.count_select(g, 3600, tm.SELECT_TRI)
    assert s2.sum() == 0 and p2.sum() == 0 and (q2 == Q).all()
    s3, p3, q3 = tm.count_select(g, 3600, tm.SELECT_STAR_PAIR | tm.SELECT_TRI)
    assert (s3 == S).all() and (p3 == P).all() and (q3 == Q).all()
    for dl in (0, 600, 86400):
        S, P, Q = oracle.count(s, d, t, dl)
        s1, p1, _ = tm.count_select(g, dl, tm.SELECT_STAR_PAIR)
        _, _, q2 = tm.count_select(g, dl, tm.SELECT_TRI)
        assert (s1 == S).all() and (p1 == P).all() and (q2 == Q).all(), dl
    deltas = [0, 60, 600, 3600, 86400, 10 ** 7]
    multi = tm.count_multi(g, deltas)
    for i, dl in enumerate(deltas):
        assert (multi[i] == tm.count(g, dl)).all(), dl
        assert (multi[i] == oracle_classes(s, d, t, dl)).all(), dl
    # monotone in delta, class by class
    assert (np.diff(multi.astype(np.int64), axis=0) >= 0).all()
    g.free()


@pytest.mark.parametrize("seed", range(4))
def test_multi_delta_single_sweep_equals_oracle(tm, seed):
    """tm_count_multi counts every window of an unsorted list with repeats in
    sweeps of up to 8 nested windows; each window must equal the oracle."""
    s, d, t = synth.random_small(700 + seed, 12, 2500, 300)
    deltas = [40, 0, 7, 300, 7, 1, 2, 150, 75, 20, 3, 500]
    g = tm.build(s, d, t)
    try:
        got = tm.count_multi(g, deltas)
        G = oracle.Graph(s, d, t)
        for i, dl in enumerate(deltas):
            want, bad = oracle.merge(*G.count(dl))
            assert bad == 0
            assert (got[i] == want).all(), (seed, dl)
    finally:
        g.free()


def test_multi_delta_on_hub_shape_equals_single_counts(tm):
    s, d, t = synth.hub(scale=0.01)
    g = tm.build(s, d, t)
    try:
        deltas = [86400, 600, 3600]
        got = tm.count_multi(g, deltas)
        for i, dl in enumerate(deltas):
            assert (got[i] == tm.count(g, dl)).all(), dl
        with pytest.raises(tm.TmError):
            tm.count_multi(g, [600, -1])
    finally:
        g.free()
