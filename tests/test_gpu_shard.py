"""Counting by shards of centres (tm_count_shard), the per-rank step of the
multi-GPU decomposition: on one GPU the shards of W ranks are counted one
after another. Each shard must equal the oracle's per-centre counters summed
over its centres, and the shards must sum (with the Tri type-I/III fill) to
the whole-graph count. Tolerance 0: the counts are integers."""
import numpy as np
import pytest

import oracle
from paper_2204_09236_gb300 import shard, synth

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


def owners(s, d, n, world):
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    own = np.zeros(n, np.int32)
    for r in range(world):
        own[shard.centre_shard(deg, world, r)] = r
    return own


def whole(tm, g, delta):
    star, pair, tri = tm.count_raw(g, delta)
    return np.concatenate([star.ravel(), pair.ravel(), tri.ravel()])


@pytest.mark.parametrize("name", ["tiny", "random"])
def test_each_shard_equals_oracle_centres(tm, name):
    if name == "tiny":
        (s, d, t), delta = synth.tiny(), 3600
    else:
        (s, d, t), delta = synth.random_small(17, 30, 3000, 400), 40
    g = tm.build(s, d, t)
    G = oracle.Graph(s, d, t)
    try:
        n = g.n
        for world in (2, 3):
            own = owners(s, d, n, world)
            for r in range(world):
                got = tm.count_shard(g, delta, own, r)
                want = np.zeros(56, np.uint64)
                for u in np.nonzero(own == r)[0]:
                    S, P, Q = G.count_centre(delta, int(u))
                    want[:24] += S.ravel()
                    want[24:32] += P.ravel()
                    want[40:48] += Q[1].ravel()  # type II; types I/III are filled after the sum
                assert (got == want).all(), (world, r)
    finally:
        g.free()


@pytest.mark.parametrize("workload", ["large", "hub"])
def test_shards_sum_to_whole_count(tm, workload):
    if workload == "large":
        (s, d, t), delta = synth.large(scale=0.01), 86400
    else:
        (s, d, t), delta = synth.hub(scale=0.01), 3600
    g = tm.build(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda())
    try:
        full = whole(tm, g, delta)
        for world in (1, 2, 5):
            own = owners(s, d, g.n, world)
            total = np.zeros(56, np.uint64)
            for r in range(world):
                total += tm.count_shard(g, delta, torch.from_numpy(own).cuda(), r)
            assert (tm.fill_tri_types(total) == full).all(), world
    finally:
        g.free()


def test_shard_rejects_bad_arguments(tm):
    s, d, t = synth.toy_graph()
    g = tm.build(s, d, t)
    try:
        with pytest.raises(ValueError):
            tm.count_shard(g, 10, np.zeros(3, np.int32), 0)
        with pytest.raises(tm.TmError):
            tm.count_shard(g, -1, np.zeros(g.n, np.int32), 0)
        # a rank that owns no centre counts nothing
        assert tm.count_shard(g, 10, np.zeros(g.n, np.int32), 1).sum() == 0
    finally:
        g.free()
