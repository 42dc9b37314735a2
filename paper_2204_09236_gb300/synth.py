"""Seeded synthetic temporal graphs shaped like the paper's workloads.

This module only draws inputs. It holds none of the counting arithmetic, and it
is the one module that both the CUDA path's tests/bench and the CPU oracle's
tests take their inputs from.

The paper measures on public SNAP / Network-Repository temporal graphs
(Section V-A, Table 2). Those datasets are not used here; each generator below
stands in for one workload shape:

* ``tiny``   - CollegeMsg scale (Table 2): 1,000 nodes, 20,000 edges, 20 % of
               them in Poisson bursts on repeated node pairs.
* ``large``  - StackOverflow scale (Table 2): 2.5M nodes, 60M edges over eight
               years with a diurnal rate, out-degree capped at 2e5.
* ``hub``    - WikiTalk-like hub skew (Fig. 8): 16 hubs of 1M incident edges
               each, 10 % exact timestamp ties.
* ``batch``  - 512 independent graphs with log-normal sizes and per-graph delta.
* ``trace``  - a Poisson request stream over batch-shaped graphs.

"Zipf(alpha)" is read as a degree power law with exponent alpha (Chung-Lu
style): node weights ``w_r = r ** (-1 / (alpha - 1))`` over ranks
``r = 1..N``, a seeded permutation maps ranks to node ids, and both endpoints
of an edge are drawn with probability proportional to the weight.

Every generator returns ``(src, dst, t)`` as numpy arrays of dtype int32,
int32, int64; edge id = array index.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2204092360
DAY = 86400
EIGHT_YEARS = 8 * 365 * DAY

# Paper's toy graph (Fig. 1), rebuilt from the edge lists printed in the
# worked examples of Section IV-A (S_a) and Section IV-B (S_e, E_(c,d)).
# Node ids: a=0, b=1, c=2, d=3, e=4.
TOY_NODES = "abcde"
TOY_EDGES = [
    ("a", "c", 4), ("a", "c", 8), ("d", "a", 9), ("a", "b", 11), ("a", "c", 15),
    ("e", "d", 1), ("e", "c", 6), ("d", "e", 14), ("e", "d", 18), ("d", "e", 21),
    ("d", "c", 10), ("c", "d", 17),
]
TOY_DELTA = 10


def toy_graph():
    src = np.array([TOY_NODES.index(a) for a, _, _ in TOY_EDGES], np.int32)
    dst = np.array([TOY_NODES.index(b) for _, b, _ in TOY_EDGES], np.int32)
    t = np.array([x for _, _, x in TOY_EDGES], np.int64)
    return src, dst, t


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


class _Zipf:
    """Draws node ids with probability proportional to a power-law weight."""

    def __init__(self, rng, ids, alpha):
        ids = np.asarray(ids, np.int64)
        r = np.arange(1, len(ids) + 1, dtype=np.float64)
        w = r ** (-1.0 / (alpha - 1.0))
        self.ids = ids[rng.permutation(len(ids))]
        self.w = w
        self._set_cdf(w)

    def _set_cdf(self, w):
        c = np.cumsum(w)
        self.cdf = c / c[-1]

    def exclude(self, mask_by_rank):
        w = self.w.copy()
        w[mask_by_rank] = 0.0
        self._set_cdf(w)

    def draw(self, rng, k):
        i = np.searchsorted(self.cdf, rng.random(k), side="right")
        return self.ids[np.minimum(i, len(self.ids) - 1)]


def _fix_self_loops(rng, z, src, dst):
    bad = np.nonzero(src == dst)[0]
    while len(bad):
        dst[bad] = z.draw(rng, len(bad))
        bad = bad[src[bad] == dst[bad]]


def _diurnal_times(rng, k, span, amp=0.5):
    """Integer seconds in [0, span) from rate 1 + amp*sin(2*pi*t/DAY).

    Inverse-CDF sampling: a uniform day, then the position inside the day by
    Newton's method on F(x) = x + amp/(2 pi) (1 - cos 2 pi x).
    """
    days = span // DAY
    d = rng.integers(0, days, size=k)
    u = rng.random(k)
    x = u.copy()
    c = amp / (2 * np.pi)
    for _ in range(30):
        f = x + c * (1 - np.cos(2 * np.pi * x)) - u
        fp = 1 + amp * np.sin(2 * np.pi * x)
        x = np.clip(x - f / fp, 0.0, 1.0 - 1e-12)
    return (d * DAY + np.floor(x * DAY)).astype(np.int64)


def tiny(seed=SEED_BASE + 1, n=1000, m=20000, burst_clusters=80, burst_len=50,
         alpha=2.1, span=1_000_000):
    rng = _rng(seed)
    z = _Zipf(rng, np.arange(n), alpha)
    nb = burst_clusters * burst_len
    mb = m - nb
    src = z.draw(rng, mb)
    dst = z.draw(rng, mb)
    _fix_self_loops(rng, z, src, dst)
    t = rng.integers(0, span, size=mb)
    bs, bd, bt = [], [], []
    for _ in range(burst_clusters):
        u = z.draw(rng, 1)[0]
        v = z.draw(rng, 1)[0]
        while v == u:
            v = z.draw(rng, 1)[0]
        s = rng.integers(0, span)
        gaps = rng.exponential(1.0, size=burst_len)
        tt = np.minimum(s + np.floor(np.cumsum(gaps)).astype(np.int64), span - 1)
        flip = rng.random(burst_len) < 0.5
        bs.append(np.where(flip, v, u))
        bd.append(np.where(flip, u, v))
        bt.append(tt)
    src = np.concatenate([src] + bs)
    dst = np.concatenate([dst] + bd)
    t = np.concatenate([t] + bt)
    relabel = rng.permutation(n)
    order = rng.permutation(m)
    return (relabel[src][order].astype(np.int32), relabel[dst][order].astype(np.int32),
            t[order].astype(np.int64))


def large(seed=SEED_BASE + 2, scale=1.0, alpha=2.0):
    """StackOverflow-shaped graph: N=2.5M, m=60M at scale 1."""
    n = max(8, int(round(2_500_000 * scale)))
    m = max(16, int(round(60_000_000 * scale)))
    cap = max(4, int(round(200_000 * scale)))
    rng = _rng(seed)
    z = _Zipf(rng, np.arange(n), alpha)
    src = z.draw(rng, m)
    # cap the out-degree: keep the first `cap` edges of a saturated source and
    # redraw the source of the rest among unsaturated nodes
    rank_of = np.empty(n, np.int64)
    rank_of[z.ids] = np.arange(n)
    while True:
        order = np.argsort(src, kind="stable")
        s = src[order]
        first = np.searchsorted(s, s, side="left")
        over = order[(np.arange(m) - first) >= cap]
        if len(over) == 0:
            break
        outdeg = np.bincount(src, minlength=n)
        z.exclude(rank_of[np.nonzero(outdeg >= cap)[0]])
        src[over] = z.draw(rng, len(over))
    z = _Zipf(_rng(seed + 1000), np.arange(n), alpha)
    rng2 = _rng(seed + 2000)
    dst = z.draw(rng2, m)
    bad = np.nonzero(src == dst)[0]
    while len(bad):
        dst[bad] = z.draw(rng2, len(bad))
        bad = bad[src[bad] == dst[bad]]
    t = _diurnal_times(rng2, m, EIGHT_YEARS)
    return src.astype(np.int32), dst.astype(np.int32), t


def hub(seed=SEED_BASE + 3, scale=1.0, n_hubs=16, alpha=2.5, tie_frac=0.10,
        span=10_000_000):
    """Hub-skew graph: N=1M, m=30M at scale 1; 16 hubs x 1M incident edges."""
    n = max(n_hubs + 8, int(round(1_000_000 * scale)))
    hub_edges = max(2, int(round(1_000_000 * scale)))
    bg = max(4, int(round(14_000_000 * scale)))
    rng = _rng(seed)
    hubs = rng.choice(n, size=n_hubs, replace=False)
    is_hub = np.zeros(n, bool)
    is_hub[hubs] = True
    z = _Zipf(rng, np.nonzero(~is_hub)[0], alpha)
    half = hub_edges // 2
    hs, hd = [], []
    for h in hubs:
        p = z.draw(rng, hub_edges)
        out = np.arange(hub_edges) < half
        hs.append(np.where(out, h, p))
        hd.append(np.where(out, p, h))
    bsrc = z.draw(rng, bg)
    bdst = z.draw(rng, bg)
    _fix_self_loops(rng, z, bsrc, bdst)
    src = np.concatenate(hs + [bsrc])
    dst = np.concatenate(hd + [bdst])
    m = len(src)
    t = rng.integers(0, span, size=m)
    # exact ties: a chosen edge copies the timestamp of another edge that is
    # incident to one of its endpoints
    k = int(round(tie_frac * m))
    chosen = rng.choice(m, size=k, replace=False)
    end = np.where(rng.random(k) < 0.5, src[chosen], dst[chosen])
    inc_node = np.concatenate([src, dst])
    inc_edge = np.concatenate([np.arange(m), np.arange(m)])
    order = np.argsort(inc_node, kind="stable")
    inc_node, inc_edge = inc_node[order], inc_edge[order]
    lo = np.searchsorted(inc_node, end, side="left")
    hi = np.searchsorted(inc_node, end, side="right")
    pick = lo + (rng.random(k) * (hi - lo)).astype(np.int64)
    t_new = t.copy()
    t_new[chosen] = t[inc_edge[pick]]
    perm = rng.permutation(m)
    return src[perm].astype(np.int32), dst[perm].astype(np.int32), t_new[perm]


BATCH_DELTAS = (60, 600, 3600, 86400)


def batch_sizes(seed=SEED_BASE + 4, count=512, lo=1_000, hi=5_000_000):
    rng = _rng(seed)
    m = np.clip(np.round(rng.lognormal(np.log(1e5), 1.2, size=count)), lo, hi)
    deltas = rng.choice(np.array(BATCH_DELTAS, np.int64), size=count)
    return m.astype(np.int64), deltas


def batch_graph(seed, m, alpha=2.1, span=1_000_000):
    m = int(m)
    n = max(3, m // 12)
    rng = _rng(seed)
    z = _Zipf(rng, np.arange(n), alpha)
    src = z.draw(rng, m)
    dst = z.draw(rng, m)
    _fix_self_loops(rng, z, src, dst)
    t = rng.integers(0, span, size=m)
    return src.astype(np.int32), dst.astype(np.int32), t.astype(np.int64)


def batch(seed=SEED_BASE + 4, count=512, scale=1.0):
    """`count` graphs of log-normal size, each with its own delta."""
    sizes, deltas = batch_sizes(seed, count)
    graphs = []
    for i, m in enumerate(sizes):
        mm = max(16, int(round(m * scale)))
        graphs.append(batch_graph(seed * 1000 + i, mm))
    return graphs, deltas


def trace(seed=SEED_BASE + 5, rate=200.0, seconds=60.0, requery=0.30):
    """Poisson request stream: (arrival_s, graph_seed or -1, graph_size, delta,
    requery_index). A re-query names no new graph; the server picks a resident
    graph with `requery_index` (uniform over residents at that moment)."""
    rng = _rng(seed)
    n = rng.poisson(rate * seconds)
    arrivals = np.sort(rng.random(n) * seconds)
    sizes, _ = batch_sizes(seed + 7, count=n)
    deltas = rng.choice(np.array(BATCH_DELTAS, np.int64), size=n)
    is_re = rng.random(n) < requery
    pick = rng.random(n)
    seeds = np.where(is_re, -1, seed * 100000 + np.arange(n))
    return arrivals, seeds, sizes, deltas, pick


def fingerprint(src, dst, t):
    """SHA-256 (hex, first 16 digits) of the three input arrays' bytes, so that
    stored results can name exactly the graph they were computed on."""
    import hashlib
    h = hashlib.sha256()
    for a, dt in ((src, np.int32), (dst, np.int32), (t, np.int64)):
        h.update(np.ascontiguousarray(a, dt).tobytes())
    return h.hexdigest()[:16]


def random_small(seed, n_nodes, m, t_range, allow_dup=True):
    """Tiny tie-heavy multigraph for brute-force checks."""
    rng = _rng(seed)
    src = rng.integers(0, n_nodes, size=m)
    dst = rng.integers(0, n_nodes - 1, size=m)
    dst = np.where(dst >= src, dst + 1, dst)
    t = rng.integers(0, t_range, size=m)
    return src.astype(np.int32), dst.astype(np.int32), t.astype(np.int64)
