"""Planted mistakes in the oracle must fail a pin.

Each case copies oracle/tm_oracle.c, plants one plausible mistake (a dropped
term, a wrong comparison, a wrong reference node, a transposed index), builds
it into a temporary library on the CPU and runs the pins of test_oracle.py
that do not depend on the planted code path. The unmodified oracle passes the
same battery.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2204_09236_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "tm_oracle.c")
GOLD = os.path.join(os.path.dirname(__file__), "golden", "toy_worked_examples.json")

MUTANTS = {
    # Algorithm 1
    "alg1_window_strict": ("if (e3.t - e1.t > delta) break;", "if (e3.t - e1.t >= delta) break;"),
    "alg1_drop_star_I_out": ("STAR(T_I, e1.dir, O, e3.dir) += h->map_out[e3.v];", ""),
    "alg1_star_III_wrong_node": ("STAR(T_III, e1.dir, IN, e3.dir) += h->map_in[e1.v];",
                                 "STAR(T_III, e1.dir, IN, e3.dir) += h->map_in[e3.v];"),
    "alg1_pair_transposed": ("PAIR(e1.dir, IN, e3.dir) += h->map_in[e1.v];",
                             "PAIR(e3.dir, IN, e1.dir) += h->map_in[e1.v];"),
    # Algorithm 2
    "alg2_raw_time_order": ("} else if (before(ei.t, ei.id, ek.t, ek.id) && before(ek.t, ek.id, ej.t, ej.id)) {",
                            "} else if (ei.t <= ek.t && ek.t <= ej.t) {"),
    "alg2_dir_k_wrt_w": ("const int dk = ek.src == v ? O : IN;", "const int dk = ek.src == w ? O : IN;"),
    "alg2_type_III_window": ("&& ek.t - ei.t <= delta) {", "&& ek.t - ej.t <= delta) {"),
    "alg2_tri_transposed": ("TRI(T_II, ei.dir, ej.dir, dk)++;", "TRI(T_II, ej.dir, ei.dir, dk)++;"),
    # the multi-threaded split (Sec. IV-C)
    "mt_chunk_end_short": ("const int64_t e = b + w->chunk < 2 * g->m ? b + w->chunk : 2 * g->m;",
                           "const int64_t e = b + w->chunk < 2 * g->m ? b + w->chunk - 1 : 2 * g->m;"),
    "mt_stale_centre": ("            while (g->off[u + 1] <= i) u++;\n", ""),
    # the definitions
    "brute_star_type": ("const int iso = s12 ? 0 : (s02 ? 1 : 2);", "const int iso = s12 ? 2 : (s02 ? 1 : 0);"),
    "brute_tri_dirk_wrt_u": ("TRI(type, dir_wrt(ei, u), dir_wrt(ej, u), dir_wrt(ek, v))++;",
                             "TRI(type, dir_wrt(ei, u), dir_wrt(ej, u), dir_wrt(ek, u))++;"),
    "brute_window_open": ("b < m && E[b].t - E[a].t <= delta; b++)\n            for (int64_t c = b + 1; c < m && E[c].t - E[a].t <= delta; c++)\n                classify_triple",
                          "b < m && E[b].t - E[a].t <= delta; b++)\n            for (int64_t c = b + 1; c < m && E[c].t - E[a].t < delta; c++)\n                classify_triple"),
}


def _battery():
    """Returns the list of failed pins."""
    failed = []
    with open(GOLD) as f:
        g = json.load(f)
    s, d, t = synth.toy_graph()
    G = oracle.Graph(s, d, t)
    star, _, _ = G.count_centre(10, 0)
    want = np.zeros((3, 2, 2, 2), np.uint64)
    T = {"I": 0, "II": 1, "III": 2}
    D = {"o": 0, "in": 1}
    for ty, a, b, c, v in g["centre_a_star"]["cells"]:
        want[T[ty], D[a], D[b], D[c]] = v
    if not (star == want).all():
        failed.append("worked example centre a")
    _, _, tri = G.count_centre(10, 4)
    want = np.zeros((3, 2, 2, 2), np.uint64)
    for ty, a, b, c, v in g["centre_e_tri"]["cells"]:
        want[T[ty], D[a], D[b], D[c]] = v
    if not (tri == want).all():
        failed.append("worked example centre e")
    for seed in range(25):
        s, d, t = synth.random_small(1000 + seed, 5, 24, 6)
        for delta in (0, 2, 4):
            a = oracle.count(s, d, t, delta)
            b = oracle.brute(s, d, t, delta)
            if not all((x == y).all() for x, y in zip(a, b)):
                failed.append("algorithms vs definition")
                break
            merged, bad = oracle.merge(*b)
            if bad or not (merged == oracle.brute_classes(s, d, t, delta)).all():
                failed.append("cells vs edge-pattern classes")
                break
        if failed:
            break
    # the multi-threaded count, with S_u lists cut into chunks
    for seed in range(6):
        s, d, t = synth.random_small(2000 + seed, 5, 30, 6)
        G = oracle.Graph(s, d, t)
        b = oracle.brute(s, d, t, 3)
        if not all((x == y).all() for x, y in zip(G.count_mt(3, threads=3, chunk=4), b)):
            failed.append("multi-threaded count vs definition")
            break
    # closed form: one static triangle counted once
    s, d, t = np.array([0, 1, 0]), np.array([1, 2, 2]), np.array([0, 1, 2])
    merged, _ = oracle.merge(*oracle.count(s, d, t, 2))
    if merged.sum() != 1:
        failed.append("single triangle")
    return failed


def _with_lib(path):
    lib = oracle._bind(ctypes.CDLL(path))
    saved = oracle._lib
    oracle._lib = lib
    try:
        return _battery()
    finally:
        oracle._lib = saved


def test_unmodified_oracle_passes_battery():
    oracle._load()
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not found: {name}"
    mutated = src.replace(old, new)
    cfile = tmp_path / "m.c"
    cfile.write_text(mutated)
    so = tmp_path / "libm.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", str(so), str(cfile)])
    assert _with_lib(str(so)) != [], f"planted mistake {name} passed every pin"
