"""Pins for the CPU oracle (no GPU).

The oracle is pinned to things other than itself:
  * the worked examples the paper prints (tests/golden/toy_worked_examples.json),
  * brute-force enumeration of the definitions (Def. 2, Def. 3) on tiny
    tie-heavy multigraphs, through two independent classifiers (counter cells
    and edge-pattern codes),
  * closed forms on pair and star graphs when delta covers the whole span,
  * invariants: relabelling, time shift, direction reversal, time reversal,
    monotonicity in delta, the isomorphism equalities of Sec. IV-A/IV-B.
"""
import json
import os
from math import comb

import numpy as np
import pytest

import oracle
from paper_2204_09236_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "toy_worked_examples.json")
T = {"I": 0, "II": 1, "III": 2}
D = {"o": 0, "in": 1}


def load_gold():
    with open(GOLD) as f:
        return json.load(f)


def graph_from(edges, nodes):
    src = np.array([nodes.index(a) for a, _, _ in edges], np.int32)
    dst = np.array([nodes.index(b) for _, b, _ in edges], np.int32)
    t = np.array([x for _, _, x in edges], np.int64)
    return src, dst, t


def motif_index(name):
    return int(name[1]) - 1, int(name[2]) - 1


# ------------------------------------------------------------ worked examples


def test_toy_graph_matches_generator():
    g = load_gold()
    s, d, t = graph_from(g["edges"], g["nodes"])
    s2, d2, t2 = synth.toy_graph()
    assert (s == s2).all() and (d == d2).all() and (t == t2).all()


def test_toy_S_lists_from_paper():
    """S_a (Sec. IV-A) and S_e (Sec. IV-B) are the time-sorted incident lists."""
    g = load_gold()
    nodes = g["nodes"]
    for centre, key in (("a", "S_a"), ("e", "S_e")):
        got = []
        for a, b, t in g["edges"]:
            if a == centre:
                got.append([t, b, "o"])
            elif b == centre:
                got.append([t, a, "in"])
        got.sort(key=lambda x: x[0])
        assert got == g[key]["entries"]
    assert nodes == "abcde"


def test_centre_a_star_worked_example():
    g = load_gold()
    s, d, t = graph_from(g["edges"], g["nodes"])
    G = oracle.Graph(s, d, t)
    star, pair, tri = G.count_centre(g["delta"], g["nodes"].index("a"))
    want = np.zeros((3, 2, 2, 2), np.uint64)
    for ty, a, b, c, v in g["centre_a_star"]["cells"]:
        want[T[ty], D[a], D[b], D[c]] = v
    assert (star == want).all()
    assert pair.sum() == 0


def test_centre_e_tri_worked_example():
    g = load_gold()
    s, d, t = graph_from(g["edges"], g["nodes"])
    G = oracle.Graph(s, d, t)
    star, pair, tri = G.count_centre(g["delta"], g["nodes"].index("e"))
    want = np.zeros((3, 2, 2, 2), np.uint64)
    for ty, a, b, c, v in g["centre_e_tri"]["cells"]:
        want[T[ty], D[a], D[b], D[c]] = v
    assert (tri == want).all()


@pytest.mark.parametrize("k", range(4))
def test_instances_printed_in_paper(k):
    g = load_gold()
    inst = g["instances"][k]
    s, d, t = graph_from(inst["edges"], g["nodes"])
    out = oracle.brute_classes(s, d, t, g["delta"])
    want = np.zeros((6, 6), np.uint64)
    want[motif_index(inst["motif"])] = 1
    assert (out == want).all()
    star, pair, tri = oracle.count(s, d, t, g["delta"])
    merged, bad = oracle.merge(star, pair, tri)
    assert bad == 0 and (merged == want).all()
    if "tri_cells" in inst:
        w = np.zeros((3, 2, 2, 2), np.uint64)
        for ty, a, b, c, v in inst["tri_cells"]:
            w[T[ty], D[a], D[b], D[c]] = v
        assert (tri == w).all()


def test_class_cells_printed_in_paper():
    g = load_gold()
    for cc in g["class_cells"]:
        i, j = motif_index(cc["motif"])
        s, p, q = oracle.class_cells(6 * i + j)
        ws, wp, wq = (np.zeros((3, 2, 2, 2), np.uint64), np.zeros((2, 2, 2), np.uint64),
                      np.zeros((3, 2, 2, 2), np.uint64))
        for ty, a, b, c in cc.get("star", []):
            ws[T[ty], D[a], D[b], D[c]] = 1
        for a, b, c in cc.get("pair", []):
            wp[D[a], D[b], D[c]] = 1
        for ty, a, b, c in cc.get("tri", []):
            wq[T[ty], D[a], D[b], D[c]] = 1
        assert (s == ws).all() and (p == wp).all() and (q == wq).all(), cc["motif"]


def test_layout_is_a_partition_of_the_56_cells():
    """Every cell belongs to exactly one class: 24 star classes of one cell,
    4 pair classes of two mirror cells, 8 triangle classes of three cells (one
    per type)."""
    S = np.zeros((3, 2, 2, 2), int)
    P = np.zeros((2, 2, 2), int)
    Q = np.zeros((3, 2, 2, 2), int)
    kinds = {"star": 0, "pair": 0, "tri": 0}
    for c in range(36):
        s, p, q = oracle.class_cells(c)
        S += s.astype(int)
        P += p.astype(int)
        Q += q.astype(int)
        ns, np_, nq = int(s.sum()), int(p.sum()), int(q.sum())
        if ns:
            assert (ns, np_, nq) == (1, 0, 0)
            kinds["star"] += 1
        elif np_:
            assert (ns, np_, nq) == (0, 2, 0)
            a, b, cc = np.argwhere(p)[0]
            assert p[1 - a, 1 - b, 1 - cc] == 1
            kinds["pair"] += 1
        else:
            assert nq == 3 and sorted(np.argwhere(q)[:, 0]) == [0, 1, 2]
            kinds["tri"] += 1
    assert (S == 1).all() and (P == 1).all() and (Q == 1).all()
    assert kinds == {"star": 24, "pair": 4, "tri": 8}


def test_full_toy_counts_consistent():
    s, d, t = synth.toy_graph()
    star, pair, tri = oracle.count(s, d, t, 10)
    bs, bp, bq = oracle.brute(s, d, t, 10)
    assert (star == bs).all() and (pair == bp).all() and (tri == bq).all()
    merged, bad = oracle.merge(star, pair, tri)
    assert bad == 0
    assert (merged == oracle.brute_classes(s, d, t, 10)).all()


# ------------------------------------------------------------- brute force


def _check_against_brute(s, d, t, delta):
    star, pair, tri = oracle.count(s, d, t, delta)
    bs, bp, bq = oracle.brute(s, d, t, delta)
    assert (star == bs).all(), (delta,)
    assert (pair == bp).all(), (delta,)
    assert (tri == bq).all(), (delta,)
    merged, bad = oracle.merge(star, pair, tri)
    assert bad == 0
    assert (merged == oracle.brute_classes(s, d, t, delta)).all()
    return merged


@pytest.mark.parametrize("seed", range(60))
def test_algorithms_equal_definition_on_tie_heavy_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 8))
    m = int(rng.integers(3, 31))
    tr = int(rng.integers(1, 12))
    s, d, t = synth.random_small(1000 + seed, n, m, tr)
    for delta in (0, 1, 2, 3, 5, 8, 100):
        _check_against_brute(s, d, t, delta)


@pytest.mark.parametrize("seed", range(6))
def test_algorithms_equal_definition_on_larger_graphs(seed):
    s, d, t = synth.random_small(5000 + seed, 12, 220, 60)
    for delta in (0, 4, 15):
        _check_against_brute(s, d, t, delta)


def test_tiny_workload_slice_against_definition():
    """A 2,000-edge slice of the tiny workload (bursts included)."""
    s, d, t = synth.tiny()
    order = np.argsort(t, kind="stable")[:2000]
    s, d, t = s[order], d[order], t[order]
    _check_against_brute(s, d, t, 3600)


def test_count_entries_partition():
    s, d, t = synth.random_small(77, 6, 40, 10)
    G = oracle.Graph(s, d, t)
    full = G.count(3)
    idx = np.arange(2 * len(s))
    rng = np.random.default_rng(0)
    rng.shuffle(idx)
    parts = [G.count_entries(3, idx[:30]), G.count_entries(3, idx[30:])]
    for k in range(3):
        assert (parts[0][k] + parts[1][k] == full[k]).all()


@pytest.mark.parametrize("seed", range(12))
def test_multithreaded_count_equals_definition(seed):
    """The hierarchical parallel count (Sec. IV-C: centres and, inside one
    S_u, ranges of first edges shared out over threads) against the
    definition, with chunks small enough to cut every S_u into pieces."""
    rng = np.random.default_rng(seed)
    s, d, t = synth.random_small(3000 + seed, int(rng.integers(3, 9)), int(rng.integers(5, 60)),
                                 int(rng.integers(1, 15)))
    G = oracle.Graph(s, d, t)
    for delta in (0, 2, 5, 100):
        want = oracle.brute(s, d, t, delta)
        for threads, chunk in ((1, 1), (2, 3), (3, 7), (5, 1 << 20)):
            got = G.count_mt(delta, threads=threads, chunk=chunk)
            for a, b in zip(got, want):
                assert (a == b).all(), (delta, threads, chunk)


def test_multithreaded_count_on_toy_and_tiny():
    s, d, t = synth.toy_graph()
    G = oracle.Graph(s, d, t)
    for threads, chunk in ((4, 1), (3, 5)):
        for a, b in zip(G.count_mt(10, threads=threads, chunk=chunk), G.count(10)):
            assert (a == b).all()
    s, d, t = synth.tiny()
    G = oracle.Graph(s, d, t)
    for a, b in zip(G.count_mt(3600, threads=4, chunk=97), G.count(3600)):
        assert (a == b).all()
    with pytest.raises(ValueError):
        G.count_mt(-1)
    with pytest.raises(ValueError):
        G.count_mt(10, chunk=0)


# ------------------------------------------------------------- closed forms


def _classes(s, d, t, delta):
    star, pair, tri = oracle.count(np.array(s), np.array(d), np.array(t), delta)
    merged, bad = oracle.merge(star, pair, tri)
    assert bad == 0
    return star, pair, tri, merged


@pytest.mark.parametrize("p,q", [(1, 1), (3, 2), (4, 5), (6, 0), (0, 5), (7, 3)])
def test_pair_closed_form(p, q):
    """p edges a->b, then q edges b->a, distinct times, delta >= span."""
    s = [0] * p + [1] * q
    d = [1] * p + [0] * q
    t = list(range(p + q))
    star, pair, tri, M = _classes(s, d, t, 10 ** 6)
    assert M[4, 4] == comb(p, 3) + comb(q, 3)  # M55: 12 12 12
    assert M[5, 5] == comb(p, 2) * q  # M66: 12 12 21
    assert M[4, 5] == p * comb(q, 2)  # M56: 12 21 21
    assert M[5, 4] == 0  # M65: 12 21 12
    assert star.sum() == 0 and tri.sum() == 0


@pytest.mark.parametrize("x,y", [(1, 1), (2, 3), (4, 2), (5, 5)])
def test_star_closed_form(x, y):
    """Centre 0: x out-edges to node 1, then y out-edges to node 2."""
    s = [0] * (x + y)
    d = [1] * x + [2] * y
    t = list(range(x + y))
    star, pair, tri, M = _classes(s, d, t, 10 ** 6)
    assert star[2, 0, 0, 0] == comb(x, 2) * y  # Star-III (o,o,o)
    assert star[0, 0, 0, 0] == x * comb(y, 2)  # Star-I (o,o,o)
    assert star[1].sum() == 0
    assert star.sum() == comb(x, 2) * y + x * comb(y, 2)
    assert M[4, 4] == comb(x, 3) + comb(y, 3)
    assert tri.sum() == 0


def test_single_triangle():
    for perm in [(0, 1, 2), (2, 0, 1), (1, 2, 0)]:
        s = np.array([0, 1, 0])[list(perm)]
        d = np.array([1, 2, 2])[list(perm)]
        star, pair, tri, M = _classes(s, d, [0, 1, 2], 2)
        assert M.sum() == 1 and tri.sum() == 3 and star.sum() == 0 and pair.sum() == 0
        assert [int(tri[k].sum()) for k in range(3)] == [1, 1, 1]
        _, _, _, M1 = _classes(s, d, [0, 1, 2], 1)
        assert M1.sum() == 0


def test_delta_zero_distinct_times_is_zero():
    s, d, _ = synth.random_small(3, 6, 40, 1)
    t = np.arange(40, dtype=np.int64) * 2
    star, pair, tri = oracle.count(s, d, t, 0)
    assert star.sum() == 0 and pair.sum() == 0 and tri.sum() == 0


def test_delta_zero_all_same_time_counts_everything():
    """delta = 0 with one shared timestamp: every triple is in the window."""
    s, d, _ = synth.random_small(4, 5, 12, 1)
    t = np.zeros(12, np.int64)
    _check_against_brute(s, d, t, 0)
    star, pair, tri = oracle.count(s, d, t, 0)
    assert star.sum() + pair.sum() + tri.sum() > 0


# ------------------------------------------------------------- invariants


def _rand(seed, n=6, m=36, tr=10):
    return synth.random_small(seed, n, m, tr)


@pytest.mark.parametrize("seed", range(5))
def test_invariant_relabel_and_shift(seed):
    s, d, t = _rand(seed)
    base = oracle.count(s, d, t, 3)
    perm = np.random.default_rng(seed).permutation(20).astype(np.int32)
    for k, x in enumerate(oracle.count(perm[s], perm[d], t + 12345, 3)):
        assert (x == base[k]).all()


@pytest.mark.parametrize("seed", range(5))
def test_invariant_direction_reversal(seed):
    s, d, t = _rand(seed)
    star, pair, tri = oracle.count(s, d, t, 4)
    rs, rp, rq = oracle.count(d, s, t, 4)
    assert (rs == star[:, ::-1, ::-1, ::-1]).all()
    assert (rp == pair[::-1, ::-1, ::-1]).all()
    assert (rq == tri[:, ::-1, ::-1, ::-1]).all()


@pytest.mark.parametrize("seed", range(5))
def test_invariant_time_reversal(seed):
    """t -> -t with edge order reversed maps (e1,e2,e3) to (e3,e2,e1):
    Star[T,a,b,c] -> Star[2-T,c,b,a], Pair[a,b,c] -> Pair[c,b,a],
    Tri[T,i,j,k] -> Tri[2-T,j,i,not k]."""
    s, d, t = _rand(seed)
    star, pair, tri = oracle.count(s, d, t, 4)
    rs, rp, rq = oracle.count(s[::-1], d[::-1], -t[::-1], 4)
    assert (rs == np.transpose(star[::-1], (0, 3, 2, 1))).all()
    assert (rp == np.transpose(pair, (2, 1, 0))).all()
    assert (rq == np.transpose(tri[::-1], (0, 2, 1, 3))[:, :, :, ::-1]).all()


@pytest.mark.parametrize("seed", range(4))
def test_invariant_monotone_in_delta(seed):
    s, d, t = _rand(seed, m=40, tr=20)
    prev = None
    for delta in range(0, 25, 3):
        _, _, _, M = _classes(s, d, t, delta)
        if prev is not None:
            assert (M >= prev).all()
        prev = M


@pytest.mark.parametrize("seed", range(4))
def test_sum_over_classes_is_number_of_small_triples(seed):
    s, d, t = _rand(seed, m=30)
    delta = 5
    _, _, _, M = _classes(s, d, t, delta)
    order = np.lexsort((np.arange(len(t)), t))
    n3 = 0
    for a in range(len(order)):
        for b in range(a + 1, len(order)):
            for c in range(b + 1, len(order)):
                ea, eb, ec = order[a], order[b], order[c]
                if t[ec] - t[ea] > delta:
                    continue
                nodes = {s[ea], d[ea], s[eb], d[eb], s[ec], d[ec]}
                n3 += len(nodes) <= 3
    assert int(M.sum()) == n3


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.Graph(np.array([0, 1]), np.array([0, 2]), np.array([1, 2]))
    with pytest.raises(ValueError):
        oracle.Graph(np.array([-1]), np.array([2]), np.array([1]))
    G = oracle.Graph(np.array([0]), np.array([1]), np.array([1]))
    with pytest.raises(ValueError):
        G.count(-1)


def test_extreme_timestamps_and_delta():
    """Window tests are differences of timestamps: no overflow near the int64
    limits, and a span beyond int64 is rejected."""
    s, d, _ = synth.random_small(6, 6, 40, 1)
    rng = np.random.default_rng(4)
    t = -(2 ** 62) + rng.integers(0, 20, size=40).astype(np.int64) * (2 ** 58)
    for delta in (0, 2 ** 58, 2 ** 60, 2 ** 63 - 1):
        _check_against_brute(s, d, t, delta)
    with pytest.raises(ValueError):
        oracle.Graph(np.array([0, 1]), np.array([1, 0]), np.array([-(2 ** 63), 2 ** 63 - 1]))


def test_empty_graph():
    G = oracle.Graph(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    star, pair, tri = G.count(5)
    assert star.sum() == 0 and pair.sum() == 0 and tri.sum() == 0


def test_fullsize_golden_files_are_complete():
    """The stored full-size cells (written by tests/golden/make_fullsize_golden.py
    from the oracle) cover every window of both workloads, and each stored cell
    set satisfies the isomorphism equalities (Sec. IV-A, IV-B)."""
    import json
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    for name, deltas in (("large", [86400]), ("hub", [600, 3600, 86400])):
        with open(os.path.join(here, f"fullsize_{name}.json")) as f:
            g = json.load(f)
        assert len(g["fingerprint"]) == 16
        assert sorted(int(k) for k in g["counts"]) == deltas
        for c in g["counts"].values():
            S = np.array(c["star"], np.uint64).reshape(3, 2, 2, 2)
            P = np.array(c["pair"], np.uint64).reshape(2, 2, 2)
            Q = np.array(c["tri"], np.uint64).reshape(3, 2, 2, 2)
            merged, bad = oracle.merge(S, P, Q)
            assert bad == 0
            assert merged.ravel().tolist() == c["classes"]
