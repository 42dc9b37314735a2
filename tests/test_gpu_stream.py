"""Incremental counting of an edge stream (tm_stream_*): time-ordered batches
appended one after another must give, after every batch, exactly the
oracle's counts of the concatenated graph so far, and each batch must add the
oracle's difference between consecutive prefixes (the instances whose last
edge is in the batch). Tolerance 0: the counts are integers."""
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


def time_ordered(s, d, t):
    o = np.argsort(t, kind="stable")
    return s[o], d[o], t[o]


def oracle_cells(s, d, t, delta):
    if len(s) == 0:
        return np.zeros(56, np.uint64)
    S, P, Q = oracle.Graph(s, d, t).count_mt(delta)
    return np.concatenate([S.ravel(), P.ravel(), Q.ravel()])


def check_stream(tm, s, d, t, delta, cuts, device=False):
    st = tm.Stream(delta)
    prev = np.zeros(56, np.uint64)
    try:
        for a, b in zip(cuts[:-1], cuts[1:]):
            bs, bd, bt = s[a:b], d[a:b], t[a:b]
            if device:
                bs, bd, bt = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (bs, bd, bt))
            added = st.append(bs, bd, bt)
            want = oracle_cells(s[:b], d[:b], t[:b], delta)
            cells, classes = st.counts()
            assert (cells == want).all(), (a, b)
            assert (added == want - prev).all(), (a, b)
            merged, bad = oracle.merge(want[:24].reshape(3, 2, 2, 2), want[24:32].reshape(2, 2, 2),
                                       want[32:].reshape(3, 2, 2, 2))
            assert bad == 0 and (classes == merged).all()
            prev = want
        assert st.edges == len(s)
        # only the edges within delta of the last timestamp stay on the device
        assert st.tail == int(np.count_nonzero(t[-1] - t <= delta))
    finally:
        st.close()


def test_tiny_in_uneven_batches(tm):
    s, d, t = time_ordered(*synth.tiny())
    # batch borders inside runs of equal timestamps (the bursts) included
    cuts = [0, 1, 2, 700, 701, 5000, 5003, 12000, 19999, 20000]
    check_stream(tm, s, d, t, 3600, cuts)


def test_batches_with_equal_timestamps_across_borders(tm):
    s, d, t = synth.random_small(91, 6, 400, 40)
    s, d, t = time_ordered(s, d, t)
    for delta in (0, 3, 50):
        check_stream(tm, s, d, t, delta, [0, 10, 11, 57, 200, 201, 399, 400])


def test_large_shape_scaled_device_batches(tm):
    s, d, t = time_ordered(*synth.large(scale=0.002))
    rng = np.random.default_rng(3)
    cuts = np.unique(np.concatenate([[0, len(s)], rng.integers(0, len(s), size=6)]))
    check_stream(tm, s, d, t, 86400, [int(x) for x in cuts], device=True)


def test_unsorted_batch_is_ordered_by_time_then_index(tm):
    s, d, t = synth.random_small(5, 5, 120, 30)
    o = np.argsort(t, kind="stable")
    first, second = o[:60], o[60:]
    second = second[::-1]  # the second batch arrives out of time order
    st = tm.Stream(7)
    try:
        st.append(s[first], d[first], t[first])
        st.append(s[second], d[second], t[second])
        # the stream's order: batch by batch, inside a batch by (t, index)
        o2 = np.concatenate([first, second[np.argsort(t[second], kind="stable")]])
        want = oracle_cells(s[o2], d[o2], t[o2], 7)
        assert (st.counts()[0] == want).all()
    finally:
        st.close()


def test_rejects_a_batch_before_the_last_timestamp(tm):
    st = tm.Stream(10)
    try:
        st.append(np.array([0, 1]), np.array([1, 2]), np.array([5, 9]))
        before = st.counts()[0].copy()
        with pytest.raises(tm.TmError) as e:
            st.append(np.array([2]), np.array([0]), np.array([8]))
        assert e.value.code == tm.TM_EINVAL
        with pytest.raises(tm.TmError):
            st.append(np.array([3]), np.array([3]), np.array([12]))  # self-loop
        assert (st.counts()[0] == before).all() and st.edges == 2
        assert st.append(np.zeros(0, np.int32), np.zeros(0, np.int32),
                         np.zeros(0, np.int64)).sum() == 0
        st.append(np.array([2]), np.array([0]), np.array([9]))  # equal to the last: allowed
        assert st.edges == 3
    finally:
        st.close()
