"""The serving loop: requests of different sizes arriving from several client
threads, continuous batching, memory-budget admission with LRU eviction, and
results that are the same alone and in the mix (tolerance 0: the counts are
integers) and equal to the oracle's counts of the same graph."""
import threading

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


def pool(k=8, scale=0.01):
    graphs, deltas = synth.batch(count=k, scale=scale)
    return list(graphs), [int(d) for d in deltas]


def alone(tm, graph, delta):
    g = tm.build(*graph)
    out = tm.count(g, delta)
    g.free()
    return out


_ORACLE = {}


def oracle_classes(key, graph, delta):
    """The oracle's 36 class counts of `graph` (literal Algorithm 1 and 2 on
    every host core), cached per (graph, delta)."""
    if (key, delta) not in _ORACLE:
        if key not in _ORACLE:
            _ORACLE[key] = oracle.Graph(*graph)
        out, bad = oracle.merge(*_ORACLE[key].count_mt(delta))
        assert bad == 0
        _ORACLE[(key, delta)] = out
    return _ORACLE[(key, delta)]


def test_results_same_alone_and_in_the_mix(tm):
    graphs, deltas = pool()
    srv = tm.Server(budget_bytes=8 << 30, workers=3, max_wave=16)
    reqs = []
    lock = threading.Lock()

    def client(c):
        rng = np.random.default_rng(c)
        for j in range(12):
            k = int(rng.integers(0, len(graphs)))
            d = int(rng.choice([60, 600, 3600, 86400]))
            if j % 3 == 0 or k % 2:
                rid = srv.submit(k, d, *graphs[k])
            else:
                rid = srv.submit(k, d, *graphs[k])  # first sight of a key carries its edges
            with lock:
                reqs.append((rid, k, d))

    threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    # re-queries of resident graphs without edges
    for k in srv.resident()[:4]:
        for d in (60, 86400):
            reqs.append((srv.submit(k, d), k, d))
    cache = {}
    for rid, k, d in reqs:
        out, lat = srv.wait(rid)
        if (k, d) not in cache:
            cache[(k, d)] = alone(tm, graphs[k], d)
        assert (out == cache[(k, d)]).all(), (rid, k, d)
        assert (out == oracle_classes(("mix", k), graphs[k], d)).all(), (rid, k, d)
        assert lat >= 0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["waves"] >= 1 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_budget_admission_and_eviction(tm):
    graphs, deltas = pool(k=6, scale=0.2)
    # the budget holds the largest graph resident beside one build, but not
    # two resident graphs and a build: new graphs must evict old ones
    est = [tm.estimate_bytes(len(g[0]), int(max(g[0].max(), g[1].max())) + 1) for g in graphs]
    budget = int(1.2 * max(r + b for r, b in est))
    srv = tm.Server(budget_bytes=budget, workers=2, max_wave=4)
    ids = [(srv.submit(k, deltas[k], *graphs[k]), k) for k in range(len(graphs))]
    for rid, k in ids:
        out, _ = srv.wait(rid)
        assert (out == alone(tm, graphs[k], deltas[k])).all()
        assert (out == oracle_classes(("budget", k), graphs[k], deltas[k])).all(), k
    st = srv.stats()
    assert st["evictions"] >= 1
    assert st["resident_bytes"] <= budget
    # an evicted key without edges is an error; a resident one is served
    gone = [k for k in range(len(graphs)) if k not in srv.resident()]
    assert gone
    with pytest.raises(tm.TmError) as e:
        srv.wait(srv.submit(gone[0], 60))
    assert e.value.code == tm.TM_EINVAL
    srv.close()


def test_graph_beyond_budget_is_rejected(tm):
    s, d, t = synth.random_small(3, 50, 20000, 1000)
    srv = tm.Server(budget_bytes=1 << 20, workers=1, max_wave=4)
    with pytest.raises(tm.TmError) as e:
        srv.wait(srv.submit(1, 10, s, d, t))
    assert e.value.code == tm.TM_EBUDGET
    srv.close()
