"""Parity at the full workload sizes, in the launch configuration bench.py
times (tm_build + whole-graph tm_count on one GPU).

  * whole graph: all 56 raw cells and the 36 classes of tm_count_raw /
    tm_count (the path bench.py times) against the oracle's cells for the same
    graph, stored in tests/golden/fullsize_*.json by
    tests/golden/make_fullsize_golden.py (literal Algorithm 1 and 2 over host
    threads; the file records the fingerprint of the input it counted, which
    the test checks before comparing);
  * sampled outputs: the per-centre counters of the CUDA path
    (tm_count_centres) against the oracle's Algorithm 1 / Algorithm 2 at the
    same centres (Star, Pair and Tri type II, which are per-centre exact), for
    a degree-stratified sample of centres;
  * properties that hold at any size: the whole-graph counts of the reversed
    graph (every edge's direction flipped) and of the time-reversed graph map
    cell by cell onto the original counts, and the pair-mirror / triangle
    triple equalities hold.
"""
import json
from pathlib import Path

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


_CACHE = {}
GOLDEN = Path(__file__).resolve().parent / "golden"


def golden(name):
    with open(GOLDEN / f"fullsize_{name}.json") as f:
        return json.load(f)


def check_golden(tm, name, deltas):
    """tm_count_raw and tm_count of the whole graph against the oracle's
    stored cells, bit for bit."""
    gold = golden(name)
    s, d, t = workload(name)
    assert synth.fingerprint(s, d, t) == gold["fingerprint"], \
        "the generator produced another graph than the one the oracle counted"
    g = tm.build(dev(s), dev(d), dev(t))
    try:
        for delta in deltas:
            want = gold["counts"][str(delta)]
            star, pair, tri = tm.count_raw(g, delta)
            assert star.ravel().tolist() == want["star"], delta
            assert pair.ravel().tolist() == want["pair"], delta
            assert tri.ravel().tolist() == want["tri"], delta
            assert tm.count(g, delta).ravel().tolist() == want["classes"], delta
    finally:
        g.free()


def workload(name):
    if name not in _CACHE:
        _CACHE[name] = synth.large() if name == "large" else synth.hub()
    return _CACHE[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def raw(tm, s, d, t, delta):
    g = tm.build(dev(s), dev(d), dev(t))
    try:
        return tm.count_raw(g, delta)
    finally:
        g.free()


def sample_centres(s, d, k_per_band=6, seed=0):
    """Centres from every degree band, skipping the few largest hubs (whose
    oracle count would take minutes)."""
    deg = np.bincount(np.concatenate([s, d]))
    rng = np.random.default_rng(seed)
    out = []
    for lo, hi in [(1, 3), (3, 10), (10, 100), (100, 1000), (1000, 20000)]:
        c = np.nonzero((deg >= lo) & (deg < hi))[0]
        if len(c):
            out += list(rng.choice(c, size=min(k_per_band, len(c)), replace=False))
    return [int(x) for x in out]


def check_invariants(tm, s, d, t, delta):
    star, pair, tri = raw(tm, s, d, t, delta)
    # isomorphic cells (Sec. IV-A, IV-B)
    assert (pair == pair[::-1, ::-1, ::-1]).all()
    cells = np.concatenate([star.ravel(), pair.ravel(), tri.ravel()])
    assert tm.merge(cells)[1] == 0
    # direction reversal: each cell goes to its o <-> in flip
    rs, rp, rq = raw(tm, d, s, t, delta)
    assert (rs == star[:, ::-1, ::-1, ::-1]).all()
    assert (rp == pair[::-1, ::-1, ::-1]).all()
    assert (rq == tri[:, ::-1, ::-1, ::-1]).all()
    # time reversal (t -> -t, edge order reversed): (e1, e2, e3) -> (e3, e2, e1)
    ts, tp, tq = raw(tm, s[::-1], d[::-1], -t[::-1], delta)
    assert (ts == np.transpose(star[::-1], (0, 3, 2, 1))).all()
    assert (tp == np.transpose(pair, (2, 1, 0))).all()
    assert (tq == np.transpose(tri[::-1], (0, 2, 1, 3))[:, :, :, ::-1]).all()
    return star, pair, tri


def check_centres(tm, s, d, t, delta, centres, key):
    if key not in _CACHE:
        _CACHE[key] = oracle.Graph(s, d, t)
    G = _CACHE[key]
    g = tm.build(dev(s), dev(d), dev(t))
    try:
        for u in centres:
            S, P, Q = G.count_centre(delta, u)
            star, pair, tri = tm.count_centres(g, delta, [u])
            assert (star == S).all(), u
            assert (pair == P).all(), u
            assert (tri[1] == Q[1]).all(), u
    finally:
        g.free()


def test_large_60M_whole_graph_equals_oracle(tm):
    check_golden(tm, "large", [86400])


@pytest.mark.parametrize("delta", sorted(int(k) for k in golden("hub")["counts"]))
def test_hub_30M_whole_graph_equals_oracle(tm, delta):
    check_golden(tm, "hub", [delta])


def test_large_60M_full_size(tm):
    s, d, t = workload("large")
    assert len(s) == 60_000_000
    check_invariants(tm, s, d, t, 86400)
    check_centres(tm, s, d, t, 86400, sample_centres(s, d), "oracle_large")


@pytest.mark.parametrize("delta", [600, 3600, 86400])
def test_hub_30M_full_size(tm, delta):
    s, d, t = workload("hub")
    assert len(s) == 30_000_000
    check_invariants(tm, s, d, t, delta)
    centres = sample_centres(s, d, k_per_band=4, seed=1)
    if delta == 600:
        # two of the 16 hubs (1M incident edges each): at delta = 600 a hub's
        # window holds about 60 entries, so the oracle's per-centre count is
        # about linear in its degree
        deg = np.bincount(np.concatenate([s, d]))
        centres += [int(u) for u in np.argsort(-deg, kind="stable")[:2]]
    check_centres(tm, s, d, t, delta, centres, "oracle_hub")
