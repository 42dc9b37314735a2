"""Writes tests/golden/fullsize_<workload>.json: the oracle's 56 raw cells and
36 class counts for the full-size large and hub workloads.

Only the oracle (oracle/, literal Algorithm 1 and Algorithm 2 spread over host
threads by ranges of first edges, Sec. IV-C) and the seeded input generators
(paper_2204_09236_gb300/synth.py) are called; no value comes from the CUDA
path. Each file records the fingerprint of the generated input, so a test
that regenerates the graph on another machine can check that it counts the
same edges.

    python tests/golden/make_fullsize_golden.py [--workload large|hub|all]
        [--threads N] [--deltas 600,3600]

Runtime on 8 x86 cores: about 10 minutes for large (delta = 86400) and about
an hour for hub (delta = 600, 3600, 86400; most of it at 86400).
"""
import argparse
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2204_09236_gb300 import synth  # noqa: E402

DELTAS = {"large": [86400], "hub": [600, 3600, 86400]}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def path_for(workload):
    return os.path.join(HERE, f"fullsize_{workload}.json")


def run(workload, threads, deltas):
    gen = synth.large if workload == "large" else synth.hub
    s, d, t = gen()
    fp = synth.fingerprint(s, d, t)
    out = {}
    p = path_for(workload)
    if os.path.exists(p):
        with open(p) as f:
            old = json.load(f)
        if old.get("fingerprint") == fp:
            out = old
    out.update({"workload": workload, "generator": f"synth.{workload}()", "m": int(len(s)),
                "fingerprint": fp,
                "note": "written by tests/golden/make_fullsize_golden.py from the oracle only"})
    out.setdefault("counts", {})
    st = time.time()
    G = oracle.Graph(s, d, t)
    build_s = time.time() - st
    for delta in deltas:
        st = time.time()
        S, P, Q = G.count_mt(delta, threads=threads)
        el = time.time() - st
        classes, bad = oracle.merge(S, P, Q)
        assert bad == 0, "isomorphic cells disagree"
        out["counts"][str(delta)] = {
            "star": [int(x) for x in S.ravel()], "pair": [int(x) for x in P.ravel()],
            "tri": [int(x) for x in Q.ravel()], "classes": [int(x) for x in classes.ravel()],
            "oracle_seconds": round(el, 1), "oracle_build_seconds": round(build_s, 1),
            "threads": threads, "cpu": cpu_model(), "machine": platform.machine()}
        with open(p, "w") as f:
            json.dump(out, f, indent=1)
        print(f"{workload} delta={delta}: {el:.1f} s on {threads} threads", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["large", "hub", "all"], default="all")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--deltas", default=None, help="comma-separated subset of the deltas")
    a = ap.parse_args()
    for wl in (["large", "hub"] if a.workload == "all" else [a.workload]):
        deltas = DELTAS[wl]
        if a.deltas:
            deltas = [x for x in deltas if str(x) in a.deltas.split(",")]
        run(wl, a.threads, deltas)


if __name__ == "__main__":
    main()
