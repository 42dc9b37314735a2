#!/usr/bin/env python
"""Throughput of exact 36-motif delta-temporal counting on one GB300.

A step is one pass of the whole path over one synthetic graph already resident
in device memory: tm_build (sort by (t, edge id), S_u for every centre, pair
lists and hash) + tm_count (Star/Pair and Tri kernels, 56 cells) + release.
value = edges / step time (device time, CUDA events on the launching stream).
e2e = the same through the public calls with pinned HOST arrays: tm_build
copies the inputs in, tm_count returns the 36 counts to the host.

Default workload: the StackOverflow-shaped large graph (2.5M nodes, 60M
edges, 8 years, delta = 86400 s). Its inputs (960 MB) exceed the 129 MB L2,
so no L2 flush is needed between steps. The same JSON line also carries
  batch: the 512-graph batched workload (build_many + count_many) next to the
         plain one-graph-per-launch path on the same graphs;
  serve: the request server on a Poisson trace (p50/p99 latency) and under a
         backlog of requests, next to the plain path serving them one by one.

--impl reference times the CPU oracle (literal Algorithm 1 and 2 on every
host core) on a bounded time-slice sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2204_09236_gb300 import synth  # noqa: E402

METRIC = "temporal edges/sec counting all 36 delta-motifs (bit-exact)"
UNIT = "edges/s"
# algorithmic bytes per edge of each timed phase (minimum a one-pass kernel
# must move): counting reads the two 16-byte incident entries of each edge
# (Star/Pair) plus the pair-list entry (Tri).
ALGO_BYTES = {"star_pair": 32, "tri": 48, "time_sort": 16, "incident": 48, "pairs": 32,
              "validate": 16}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one count's Tri
# phase (k_tri_jobs + k_tri_join) from one ncu capture, with the SHA-256
# prefix of csrc/count.cu the capture ran and the command that made it. A
# count.cu that differs from the captured one reports null traffic.
PHASE_TRAFFIC = {}

WORKLOADS = {
    "large": dict(desc="large: 2.5M nodes, 60M edges, Zipf(2.0) degree law, out-degree cap 2e5, "
                       "8 years, diurnal rate", delta=86400),
    "hub": dict(desc="hub: 1M nodes, 30M edges, 16 hubs x 1M edges, Zipf(2.5), 1e7 s, "
                     "10% exact ties", delta=3600),
    "tiny": dict(desc="tiny: 1,000 nodes, 20,000 edges, Zipf(2.1), 20% bursts, 1e6 s",
                 delta=3600),
    "serve": dict(desc="serving", delta=None),
    "batch": dict(desc="batch: 512 graphs, m ~ LogNormal(ln 1e5, 1.2) clipped to [1e3, 5e6], "
                       "N = m/12, Zipf(2.1), 1e6 s, per-graph delta in {60, 600, 3600, 86400}",
                  delta=None),
}


def count_cu_sha():
    with open(os.path.join(ROOT, "paper_2204_09236_gb300", "csrc", "count.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def phase_traffic(workload, scale, phase):
    rec = PHASE_TRAFFIC.get((workload, phase))
    if rec is None or scale != 1.0 or rec["count_cu"] != count_cu_sha():
        return None
    return rec["bytes"]


def gen_batch(scale, seed_offset, count=512):
    cache = os.path.join(tempfile.gettempdir(), f"tm_bench_batch_{scale}_{seed_offset}_{count}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        m = z["m"]
        offs = np.concatenate([[0], np.cumsum(m)])
        graphs = [(z["s"][offs[i]:offs[i + 1]], z["d"][offs[i]:offs[i + 1]],
                   z["t"][offs[i]:offs[i + 1]]) for i in range(len(m))]
        return graphs, z["deltas"]
    graphs, deltas = synth.batch(seed=synth.SEED_BASE + 4 + seed_offset, count=count, scale=scale)
    try:
        np.savez(cache, s=np.concatenate([g[0] for g in graphs]),
                 d=np.concatenate([g[1] for g in graphs]), t=np.concatenate([g[2] for g in graphs]),
                 m=np.array([len(g[0]) for g in graphs]), deltas=np.asarray(deltas))
    except OSError:
        pass
    return graphs, deltas


def gen(workload, scale, seed_offset):
    key = f"{workload}_{scale}_{seed_offset}"
    cache = os.path.join(tempfile.gettempdir(), f"tm_bench_{key}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        return z["s"], z["d"], z["t"]
    if workload == "large":
        s, d, t = synth.large(seed=synth.SEED_BASE + 2 + seed_offset, scale=scale)
    elif workload == "hub":
        s, d, t = synth.hub(seed=synth.SEED_BASE + 3 + seed_offset, scale=scale)
    else:
        s, d, t = synth.tiny(seed=synth.SEED_BASE + 1 + seed_offset)
    try:
        np.savez(cache, s=s, d=d, t=t)
    except OSError:
        pass
    return s, d, t


class Clocks:
    """Samples nvidia-smi every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def timed_wall(fn, steps, warmup, torch, dist=None):
    """Wall time per call of fn (synchronous calls), after warm-up."""
    out = None
    for _ in range(warmup):
        out = fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = time.perf_counter()
    for _ in range(steps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - st) / max(steps, 1), out


def measure_batch(tm, torch, graphs, deltas, steps, warmup, tune, dist=None):
    """Many graphs in one batched count (tm_build_many + tm_count_many) vs
    one graph per launch (tm_build + tm_count per graph), inputs resident on
    the device; the two must give identical counts."""
    deltas = [int(x) for x in deltas]
    ms = np.array([len(g[0]) for g in graphs], np.int64)
    M = int(ms.sum())
    offs = np.concatenate([[0], np.cumsum(ms)])
    s_all = torch.from_numpy(np.concatenate([g[0] for g in graphs])).cuda()
    d_all = torch.from_numpy(np.concatenate([g[1] for g in graphs])).cuda()
    t_all = torch.from_numpy(np.concatenate([g[2] for g in graphs])).cuda()
    views = [(s_all[offs[i]:offs[i + 1]], d_all[offs[i]:offs[i + 1]], t_all[offs[i]:offs[i + 1]])
             for i in range(len(graphs))]
    torch.cuda.synchronize()

    def batched():
        g = tm.build_many(views)
        out = tm.count_many(g, deltas)
        g.free()
        return out

    def plain():
        outs = []
        for v, dl in zip(views, deltas):
            g = tm.build(*v)
            outs.append(tm.count(g, dl))
            g.free()
        return np.stack(outs)

    tuned = None
    if tune:
        g = tm.build_many(views)
        ie, bps, tms = tm.tune_batch(g, deltas, reps=1)
        g.free()
        tuned = {"item_entries": ie, "blocks_per_sm": bps, "count_ms": tms}
    l0 = tm.launch_count()
    step, out_b = timed_wall(batched, steps, warmup, torch, dist)
    launches = (tm.launch_count() - l0) / max(steps + warmup, 1)
    g = tm.build_many(views)
    c_step, _ = timed_wall(lambda: tm.count_many(g, deltas), steps, 1, torch)
    g.free()
    p_step, out_p = timed_wall(plain, max(1, steps // 2), 1, torch)
    built = [tm.build(*v) for v in views]
    pc_step, _ = timed_wall(lambda: [tm.count(h, dl) for h, dl in zip(built, deltas)],
                            max(1, steps // 2), 1, torch)
    for h in built:
        h.free()
    return {"graphs": len(graphs), "m_total": M, "value": M / step, "unit": UNIT,
            "ms": step * 1e3, "count_only": {"value": M / c_step, "unit": UNIT, "ms": c_step * 1e3},
            "plain_one_graph_per_launch": {"value": M / p_step, "unit": UNIT, "ms": p_step * 1e3,
                                           "count_only": {"value": M / pc_step, "unit": UNIT,
                                                          "ms": pc_step * 1e3}},
            "speedup_vs_plain": p_step / step, "batched_equals_plain": bool((out_b == out_p).all()),
            "launches_per_step": launches, "tune": tuned, "batch_config": tm.batch_get_config(),
            "timing": "wall clock around synchronous calls, inputs resident on the device"}


def serve_trace(tm, srv, pool, rate, seconds, saturate):
    """Replays a Poisson trace of requests on srv: 70% new graphs (cycling
    through `pool`), 30% re-queries of resident graphs with a new delta. With
    `saturate` every request is submitted at once (a backlog) and re-queries
    name an earlier graph with its edges. Returns (submitted requests,
    latencies, wall seconds)."""
    arrivals, seeds, _, deltas, pick = synth.trace(rate=rate, seconds=seconds)
    reqs = []
    next_key = 0
    start = time.perf_counter()
    for i in range(len(arrivals)):
        if not saturate:
            now = time.perf_counter() - start
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
        d = int(deltas[i])
        if seeds[i] < 0 and next_key > 0:
            if saturate:
                key = int(pick[i] * next_key) % next_key
                reqs.append((srv.submit(key, d, *pool[key % len(pool)]), key, d))
                continue
            res = srv.resident()
            if res:
                key = res[int(pick[i] * len(res)) % len(res)]
                reqs.append((srv.submit(key, d), key, d))
                continue
        reqs.append((srv.submit(next_key, d, *pool[next_key % len(pool)]), next_key, d))
        next_key += 1
    lat, outs = [], []
    for rid, key, d in reqs:
        out, l = srv.wait(rid, timeout=600)
        lat.append(l)
        outs.append(out)
    wall = time.perf_counter() - start
    return reqs, outs, np.sort(np.array(lat)), wall


def measure_serve(tm, pool, args, local):
    """The server on a Poisson trace (latency) and under a backlog
    (throughput) next to the plain path serving the backlog's requests one by
    one (tm_build for a new graph, tm_count for every request)."""
    budget = int(args.budget_gb * (1 << 30))
    res = {"config": {"workload": f"Poisson {args.rate} req/s for {args.seconds} s; backlog of "
                                  f"{args.sat_seconds * args.rate:.0f} requests; pool of {len(pool)} "
                                  "batch-shaped graphs; 70% new graphs, 30% re-queries with a new "
                                  "delta", "budget_gb": args.budget_gb,
                      "workers": args.serve_workers, "max_wave": args.serve_wave}}
    srv = tm.Server(budget_bytes=budget, workers=args.serve_workers, max_wave=args.serve_wave)
    srv.wait(srv.submit(-1, 600, *pool[0]))  # warm-up: plans, streams, kernels
    with Clocks(local) as clk:
        reqs, outs, lat, wall = serve_trace(tm, srv, pool, args.rate, args.seconds, False)
    st = srv.stats()
    srv.close()
    res["poisson"] = {"value": len(reqs) / wall, "unit": "requests/s",
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "max_ms": float(lat[-1]), "edges_per_s": st["edges_counted"] / wall,
                      "requests": len(reqs), "server": st, "clocks": clk.summary()}
    # backlog: the server against the plain path on the same requests
    srv = tm.Server(budget_bytes=budget, workers=args.serve_workers, max_wave=args.serve_wave)
    srv.wait(srv.submit(-1, 600, *pool[0]))
    reqs, outs, lat, wall = serve_trace(tm, srv, pool, args.rate, args.sat_seconds, True)
    st = srv.stats()
    srv.close()
    built = {}
    start = time.perf_counter()
    plain_outs = []
    for _, key, d in reqs:
        if key not in built:
            built[key] = tm.build(*pool[key % len(pool)])
        plain_outs.append(tm.count(built[key], d))
    plain_wall = time.perf_counter() - start
    for g in built.values():
        g.free()
    edges = sum(len(pool[k % len(pool)][0]) for _, k, _ in reqs)
    res["backlog"] = {"value": len(reqs) / wall, "unit": "requests/s", "edges_per_s": edges / wall,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "plain_one_request_at_a_time": {"value": len(reqs) / plain_wall,
                                                      "unit": "requests/s",
                                                      "edges_per_s": edges / plain_wall},
                      "speedup_vs_plain": plain_wall / wall, "requests": len(reqs),
                      "served_equals_alone": bool(all((a == b).all()
                                                      for a, b in zip(outs, plain_outs))),
                      "server": st}
    return res


def time_slice(s, d, t, days):
    t0 = int(t.min())
    sel = t < t0 + days * 86400
    return s[sel], d[sel], t[sel]


def oracle_run(s, d, t, delta, threads):
    """Oracle build + literal Algorithm 1 and 2 (spread over `threads` host
    threads by ranges of first edges); returns the seconds it took."""
    import oracle
    st = time.perf_counter()
    G = oracle.Graph(s, d, t)
    if threads == 1:
        G.count(delta)
    else:
        G.count_mt(delta, threads=threads)
    return time.perf_counter() - st


def cpu_baseline(s, d, t, delta, days):
    """The oracle on every host core, on the edges of the first `days` days
    of the workload (a bounded sample: a few seconds to tens of seconds)."""
    ss, dd, tt = time_slice(s, d, t, days)
    cores = os.cpu_count() or 1
    el = oracle_run(ss, dd, tt, delta, cores)
    return {"value": len(ss) / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"first {days} days of the same workload ({len(ss)} edges, delta={delta}); "
                      f"oracle build + Algorithm 1 + Algorithm 2 on {cores} threads, {el:.1f} s"}


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step counts the bounded time
    slice of the workload on all host cores (rank 0 only)."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    delta = args.delta if args.delta is not None else wl["delta"]
    s, d, t = gen(args.workload, args.scale, 0)
    import oracle
    oracle.build()
    days = args.cpu_sample_days
    ss, dd, tt = time_slice(s, d, t, days)
    cores = os.cpu_count() or 1
    times = []
    for k in range(args.warmup + args.steps):
        el = oracle_run(ss, dd, tt, delta, cores)
        if k >= args.warmup:
            times.append(el)
    step = sum(times) / len(times)
    v = len(ss) / step
    sample = (f"first {days} days of the {args.workload} workload ({len(ss)} edges) per step, "
              f"oracle build + Algorithm 1 + Algorithm 2 on {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": wl["desc"], "delta": delta, "m": len(ss)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def measure_single(tm, torch, args, s, d, t, delta, world, dist, local):
    """The step (build + count + release) on the device-resident graph, the
    count alone, the phase timers and the end-to-end calls from host arrays."""
    m = len(s)
    src = torch.from_numpy(s).cuda()
    dst = torch.from_numpy(d).cuda()
    tt = torch.from_numpy(t).cuda()
    cells = torch.zeros(56, dtype=torch.uint64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        g = tm.build_async(src, dst, tt, stream)
        tm.count_async(g, delta, cells, stream)
        g.free_async(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    tm.tm_profile_read()
    tm.tm_profile_enable(True)
    l0 = tm.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    tm.tm_profile_enable(False)
    launches = tm.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    phases = tm.tm_profile_read()
    if dist:
        x = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        ms = float(x.item())
    out = {"ms_step": ms / args.steps, "launches": launches, "clocks": clk.summary(),
           "phases": {k: v[0] / max(v[1], 1) for k, v in phases.items()}}
    count_ms = None
    if not args.no_count_only:
        g = tm.build_async(src, dst, tt, stream)
        for _ in range(2):
            tm.count_async(g, delta, cells, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            tm.count_async(g, delta, cells, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        count_ms = e0.elapsed_time(e1) / args.steps
        g.free_async(stream)
        torch.cuda.synchronize()
    out["count_ms"] = count_ms
    out["cells"] = cells.cpu().numpy()
    del src, dst, tt
    out["e2e"] = None
    if not args.no_e2e:
        hs = torch.from_numpy(s).pin_memory()
        hd = torch.from_numpy(d).pin_memory()
        ht = torch.from_numpy(t).pin_memory()
        for _ in range(max(1, args.warmup)):
            g = tm.build(hs, hd, ht)
            tm.count(g, delta)
            g.free()
        times = []
        for _ in range(args.steps):
            st = time.perf_counter()
            g = tm.build(hs, hd, ht)
            tm.count(g, delta)
            g.free()
            times.append(time.perf_counter() - st)
        e2e_step = sum(times) / len(times)
        if dist:
            x = torch.tensor([e2e_step], device="cuda", dtype=torch.float64)
            dist.all_reduce(x, op=dist.ReduceOp.MAX)
            e2e_step = float(x.item())
        out["e2e"] = {"value": world * m / e2e_step, "unit": UNIT, "h2d_bytes_per_step": 16 * m,
                      "d2h_bytes_per_step": 36 * 8, "ms_per_step": e2e_step * 1e3}
    return out


def measure_shard(tm, torch, args, s, d, t, delta, world, rank, dist):
    """Strong scaling of the count over ranks: every rank builds the whole
    graph, counts the centres of its shard (tm_count_shard) and the 56 cells
    are summed over the ranks (one all-reduce) and filled; timed: the count,
    the all-reduce and the fill, max over ranks."""
    from paper_2204_09236_gb300 import shard
    g = tm.build(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda())
    deg = np.bincount(np.concatenate([s, d]), minlength=g.n)
    own = np.zeros(g.n, np.int32)
    for r in range(world):
        own[shard.centre_shard(deg, world, r)] = r
    own_d = torch.from_numpy(own).cuda()

    def step():
        cells = tm.count_shard(g, delta, own_d, rank)
        return tm.fill_tri_types(shard.all_reduce_cells(cells, dist))

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = time.perf_counter()
    for _ in range(args.steps):
        out = step()
    torch.cuda.synchronize()
    el = (time.perf_counter() - st) / args.steps
    if dist:
        x = torch.tensor([el], device="cuda", dtype=torch.float64)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        el = float(x.item())
    whole = tm.count_raw(g, delta)
    same = bool((out == np.concatenate([a.ravel() for a in whole])).all())
    g.free()
    return el, same


def measure_hub(tm, torch, steps):
    """The hub-skew workload at its three windows: the step (build + count)
    per delta, the count alone, and tm_count_multi over the three windows
    against three separate tm_count calls (graph resident, wall clock around
    the synchronous calls)."""
    deltas = [600, 3600, 86400]
    s, d, t = gen("hub", 1.0, 0)
    m = len(s)
    src, dst, tt = (torch.from_numpy(x).cuda() for x in (s, d, t))
    stream = torch.cuda.current_stream()
    cells = torch.zeros(56, dtype=torch.uint64, device="cuda")
    out = {"workload": WORKLOADS["hub"]["desc"], "m": m, "per_delta": {}}
    for delta in deltas:
        def step():
            g = tm.build_async(src, dst, tt, stream)
            tm.count_async(g, delta, cells, stream)
            g.free_async(stream)
        for _ in range(2):
            step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / steps
        g = tm.build_async(src, dst, tt, stream)
        tm.count_async(g, delta, cells, stream)
        e0.record(stream)
        for _ in range(steps):
            tm.count_async(g, delta, cells, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        count_ms = e0.elapsed_time(e1) / steps
        g.free_async(stream)
        out["per_delta"][str(delta)] = {"value": m / (step_ms / 1e3), "unit": UNIT,
                                        "step_ms": step_ms, "count_ms": count_ms,
                                        "count_only": m / (count_ms / 1e3)}
    g = tm.build(src, dst, tt)
    multi_ms, multi = timed_wall(lambda: tm.count_multi(g, deltas), steps, 1, torch)
    sep_ms, sep = timed_wall(lambda: np.stack([tm.count(g, x) for x in deltas]), steps, 1, torch)
    g.free()
    out["multi_delta"] = {"deltas": deltas, "multi_ms": multi_ms * 1e3,
                          "separate_ms": sep_ms * 1e3, "speedup": sep_ms / multi_ms,
                          "multi_equals_separate": bool((multi == sep).all()),
                          "timing": "wall clock around synchronous calls, graph resident"}
    return out


def roofline_of(phases, m, workload, scale):
    peak, peak_kind = measured_peak()

    def gbs(phase):
        return ALGO_BYTES[phase] * m / (phases[phase] / 1e3) / 1e9 if phases.get(phase) else None

    achieved = gbs("tri")
    return {"bound": "hbm", "kernel": "tri phase: k_tri_jobs + k_tri_join",
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
            "traffic": phase_traffic(workload, scale, "tri"),
            "algo_bytes_per_edge": ALGO_BYTES["tri"], "kernel_ms": phases.get("tri"),
            "phases": {k: {"ms": round(phases[k], 4), "algo_GBps": round(gbs(k), 1),
                           "frac": round(gbs(k) / peak, 4)} for k in phases if phases[k] > 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--delta", type=int, default=None)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-sample-days", type=int, default=120)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-count-only", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch object of the line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serve object of the line")
    ap.add_argument("--no-hub", action="store_true", help="skip the hub object of the line")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch: skip the autotuner (use the library defaults)")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--shard", action="store_true",
                    help="count one graph split by centres over the ranks (strong scaling)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: requests per second")
    ap.add_argument("--seconds", type=float, default=None,
                    help="serve: Poisson trace length (60 for --workload serve, else 10)")
    ap.add_argument("--sat-seconds", type=float, default=5.0,
                    help="serve: backlog = rate x sat-seconds requests submitted at once")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: device budget")
    ap.add_argument("--serve-pool", type=int, default=96, help="serve: distinct new graphs")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-wave", type=int, default=64)
    args = ap.parse_args()
    if args.seconds is None:
        args.seconds = 60.0 if args.workload == "serve" else 10.0

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2204_09236_gb300 import tm
    common = {"n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "int64",
              "data": "synthetic (seeded generators standing in for the paper's SNAP datasets)"}

    if args.workload == "batch":
        graphs, deltas = gen_batch(args.scale, rank)
        with Clocks(local) as clk:
            b = measure_batch(tm, torch, graphs, deltas, args.steps, args.warmup, not args.no_tune,
                              dist)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": world * b["value"], "unit": UNIT,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms"],
                              **common, "config": {"workload": WORKLOADS["batch"]["desc"],
                                                   "scale": args.scale}, "batch": b,
                              "clocks": clk.summary()}))
    elif args.workload == "serve":
        pool, _ = gen_batch(args.scale, 0, count=args.serve_pool)
        sv = measure_serve(tm, list(pool), args, local)
        if rank == 0:
            print(json.dumps({"metric": "serving: requests/s with p50/p99 latency (exact 36-motif "
                                        "counts)", "value": sv["poisson"]["value"],
                              "unit": "requests/s", "steps": 1, "warmup": 1, **common,
                              "config": sv["config"], "serve": sv}))
    elif args.shard:
        wl = WORKLOADS[args.workload]
        delta = args.delta if args.delta is not None else wl["delta"]
        s, d, t = gen(args.workload, args.scale, 0)
        with Clocks(local) as clk:
            el, same = measure_shard(tm, torch, args, s, d, t, delta, world, rank, dist)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": len(s) / el, "unit": UNIT, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": el * 1e3, **common, "scaling": "strong",
                "config": {"workload": wl["desc"], "m": len(s), "delta": delta,
                           "parallelism": f"centre shards over {world} ranks, graph replicated, "
                                          "one all-reduce of 56 cells",
                           "timed": "tm_count_shard + all-reduce + type fill (graph resident)"},
                "shards_sum_to_whole_count": same, "clocks": clk.summary()}))
    else:
        wl = WORKLOADS[args.workload]
        delta = args.delta if args.delta is not None else wl["delta"]
        # every rank counts its own independent graph (weak scaling, no exchange)
        s, d, t = gen(args.workload, args.scale, rank)
        m = len(s)
        r = measure_single(tm, torch, args, s, d, t, delta, world, dist, local)
        _, bad = tm.merge(r["cells"])
        cpu = None
        if rank == 0 and not args.no_cpu_baseline:
            cpu = cpu_baseline(s, d, t, delta, args.cpu_sample_days)
        del s, d, t
        batch = serve = hub = None
        if rank == 0 and not args.no_hub and args.workload == "large":
            hub = measure_hub(tm, torch, args.steps)
        if rank == 0 and not args.no_batch:
            graphs, deltas = gen_batch(1.0, 0)
            batch = measure_batch(tm, torch, graphs, deltas, args.batch_steps, 1,
                                  not args.no_tune)
            batch["config"] = WORKLOADS["batch"]["desc"]
            del graphs
        if rank == 0 and not args.no_serve:
            pool, _ = gen_batch(1.0, 0, count=args.serve_pool)
            serve = measure_serve(tm, list(pool), args, local)
        if rank == 0:
            ms_step = r["ms_step"]
            print(json.dumps({
                "metric": METRIC, "value": world * m / (ms_step / 1e3), "unit": UNIT,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, **common,
                "config": {"workload": wl["desc"], "m": m, "delta": delta, "scale": args.scale,
                           "l2": "inputs (16 B/edge) larger than the 129 MB L2; no flush",
                           "parallelism": f"replicas{world}" if world > 1 else "single"},
                "e2e": r["e2e"], "roofline": roofline_of(r["phases"], m, args.workload, args.scale),
                "cpu_baseline": cpu, "clocks": r["clocks"], "gpu_launches": r["launches"],
                "count_only": ({"value": m / (r["count_ms"] / 1e3), "unit": UNIT,
                                "ms": r["count_ms"]} if r["count_ms"] else None),
                "phases_ms": {k: round(v, 4) for k, v in r["phases"].items()},
                "isomorphism_mismatches": bad, "hub": hub, "batch": batch, "serve": serve}))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
