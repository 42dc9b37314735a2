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
so no L2 flush is needed between steps.

--impl reference times the CPU oracle (literal Algorithm 1 and 2, one host
thread) on a bounded time-slice sample of the same workload.
"""
import argparse
import json
import os
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

# DRAM bytes (read + write) of the Tri phase (k_tri_jobs + k_tri_join) on the
# full workload, from one ncu capture of dram__bytes_read.sum +
# dram__bytes_write.sum (profiles/count_kernels_dram_large_60M.md); None until
# captured for the current kernels
TRI_TRAFFIC = {"large": 9.06e9 + 0.302e9 + 4.00e9 + 0.084e9}

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


def gen_batch(scale, seed_offset):
    cache = os.path.join(tempfile.gettempdir(), f"tm_bench_batch_{scale}_{seed_offset}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        m = z["m"]
        offs = np.concatenate([[0], np.cumsum(m)])
        graphs = [(z["s"][offs[i]:offs[i + 1]], z["d"][offs[i]:offs[i + 1]],
                   z["t"][offs[i]:offs[i + 1]]) for i in range(len(m))]
        return graphs, z["deltas"]
    graphs, deltas = synth.batch(seed=synth.SEED_BASE + 4 + seed_offset, scale=scale)
    try:
        np.savez(cache, s=np.concatenate([g[0] for g in graphs]),
                 d=np.concatenate([g[1] for g in graphs]), t=np.concatenate([g[2] for g in graphs]),
                 m=np.array([len(g[0]) for g in graphs]), deltas=np.asarray(deltas))
    except OSError:
        pass
    return graphs, deltas


def run_serve(args, rank, world, dist):
    """Poisson request stream: new graphs drawn as in the batched workload and
    re-queries of resident graphs with a new delta, served with continuous
    batching under a device-memory budget; p50/p99 latency and throughput."""
    import torch
    from paper_2204_09236_gb300 import tm
    pool, _ = synth.batch(count=args.serve_pool, scale=args.scale)
    pool = list(pool)
    arrivals, seeds, _, deltas, pick = synth.trace(rate=args.rate, seconds=args.seconds)
    srv = tm.Server(budget_bytes=int(args.budget_gb * (1 << 30)), workers=args.serve_workers,
                    max_wave=args.serve_wave)
    # warm-up: one request so that plans, streams and kernels are loaded
    srv.wait(srv.submit(-1, 600, *pool[0]))
    ids = []
    next_key = 0
    start = time.perf_counter()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for i in range(len(arrivals)):
            now = time.perf_counter() - start
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            res = srv.resident() if seeds[i] < 0 else []
            if res:
                key = res[int(pick[i] * len(res)) % len(res)]
                ids.append((srv.submit(key, int(deltas[i])), key, int(deltas[i]), None))
            else:
                g = pool[next_key % len(pool)]
                ids.append((srv.submit(next_key, int(deltas[i]), *g), next_key, int(deltas[i]),
                            next_key % len(pool)))
                next_key += 1
        lat = []
        outs = {}
        for rid, key, d, pj in ids:
            out, l = srv.wait(rid, timeout=600)
            lat.append(l)
            if pj is not None:
                outs[(pj, d)] = out
        wall = time.perf_counter() - start
    st = srv.stats()
    srv.close()
    # determinism: a sample of served results against the same graph counted alone
    rng = np.random.default_rng(0)
    sample = list(outs.items())
    rng.shuffle(sample)
    same = True
    for (pj, d), out in sample[:args.serve_check]:
        g = tm.build(*pool[pj])
        same &= bool((tm.count(g, d) == out).all())
        g.free()
    lat = np.sort(np.array(lat))
    if rank == 0:
        print(json.dumps({
            "metric": "serving: requests/s with p50/p99 latency (exact 36-motif counts)",
            "value": len(ids) / wall, "unit": "requests/s", "n_gpus": world, "steps": 1,
            "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"serving: Poisson {args.rate} req/s for {args.seconds} s, 70% new "
                                   f"graphs (drawn from a pool of {len(pool)} batch-shaped graphs), "
                                   "30% re-queries of resident graphs with a new delta",
                       "budget_gb": args.budget_gb, "workers": args.serve_workers,
                       "max_wave": args.serve_wave, "scale": args.scale},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat[-1]), "edges_per_s": st["edges_counted"] / wall,
            "server": st, "served_equals_alone": same, "checked": min(len(sample), args.serve_check),
            "clocks": clk.summary()}))


def run_batch(args, rank, world, dist):
    """Many graphs in one persistent launch vs one graph per launch."""
    import torch
    from paper_2204_09236_gb300 import tm
    graphs, deltas = gen_batch(args.scale, rank)
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

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            out = fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        st = time.perf_counter()
        for _ in range(steps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - st) / steps, out

    tune = None
    if not args.no_tune:
        g = tm.build_many(views)
        ie, bps, tms = tm.tune_batch(g, deltas, reps=2)
        g.free()
        tune = {"item_entries": ie, "blocks_per_sm": bps, "count_ms": tms}
    l0 = tm.launch_count()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        step, out_b = timed(batched, args.steps, args.warmup)
    launches = tm.launch_count() - l0
    # count only, the graph resident
    g = tm.build_many(views)
    c_step, _ = timed(lambda: tm.count_many(g, deltas), args.steps, 1)
    g.free()
    p_step, out_p = timed(plain, max(1, args.steps // 2), 1)
    same = bool((out_b == out_p).all())
    if dist:
        x = torch.tensor([step, p_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        step, p_step = float(x[0]), float(x[1])
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": world * M / step, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded generators standing in for the paper's SNAP datasets)",
            "config": {"workload": WORKLOADS["batch"]["desc"], "graphs": len(graphs), "m_total": M,
                       "scale": args.scale, "timing": "wall clock around synchronous calls"},
            "count_only": {"value": M / c_step, "unit": UNIT, "ms": c_step * 1e3},
            "plain_one_graph_per_launch": {"value": M / p_step, "unit": UNIT, "ms": p_step * 1e3},
            "batched_equals_plain": same, "tune": tune, "clocks": clk.summary(),
            "gpu_launches": launches, "batch_config": tm.batch_get_config()}))


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


def cpu_baseline(s, d, t, delta, days, timeout_s=60.0):
    """The oracle (single host thread) on the edges of the first `days` days."""
    import oracle
    t0 = int(t.min())
    sel = t < t0 + days * 86400
    ss, dd, tt = s[sel], d[sel], t[sel]
    start = time.perf_counter()
    G = oracle.Graph(ss, dd, tt)
    G.count(delta)
    el = time.perf_counter() - start
    return {"value": len(ss) / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {days} days of the same workload ({len(ss)} edges, delta={delta}); "
                      f"oracle build + Algorithm 1 + Algorithm 2, {el:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    delta = args.delta if args.delta is not None else wl["delta"]
    s, d, t = gen(args.workload, args.scale, 0)
    import oracle
    oracle.build()
    days = args.cpu_sample_days
    t0 = int(t.min())
    sel = t < t0 + days * 86400
    ss, dd, tt = s[sel], d[sel], t[sel]
    times = []
    for k in range(args.warmup + args.steps):
        st = time.perf_counter()
        G = oracle.Graph(ss, dd, tt)
        G.count(delta)
        el = time.perf_counter() - st
        if k >= args.warmup:
            times.append(el)
    step = sum(times) / len(times)
    v = len(ss) / step
    sample = f"first {days} days of the {args.workload} workload ({len(ss)} edges) per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": wl["desc"], "delta": delta, "m": len(ss)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--delta", type=int, default=None)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-sample-days", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-count-only", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch workload: skip the autotuner (use the library defaults)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: requests per second")
    ap.add_argument("--seconds", type=float, default=60.0, help="serve: trace length")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: device budget")
    ap.add_argument("--serve-pool", type=int, default=96, help="serve: distinct new graphs")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-wave", type=int, default=64)
    ap.add_argument("--serve-check", type=int, default=24)
    args = ap.parse_args()

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

    if args.workload in ("batch", "serve"):
        (run_batch if args.workload == "batch" else run_serve)(args, rank, world, dist)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    wl = WORKLOADS[args.workload]
    delta = args.delta if args.delta is not None else wl["delta"]
    # every rank counts its own independent graph (weak scaling, no exchange)
    s, d, t = gen(args.workload, args.scale, rank)
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
    ms_step = ms / args.steps
    value = world * m / (ms_step / 1e3)

    # per-phase device times (events on the launching stream, one pair per
    # phase and step); the Tri join kernel is the largest single kernel of
    # the step (profiles/launch_list_large_60M.md)
    ph = {k: v[0] / max(v[1], 1) for k, v in phases.items()}
    peak, peak_kind = measured_peak()

    def gbs(phase):
        return ALGO_BYTES[phase] * m / (ph[phase] / 1e3) / 1e9 if ph.get(phase) else None

    achieved = gbs("tri")
    roofline = {"bound": "hbm", "kernel": "tri phase: k_tri_jobs + k_tri_join",
                "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": TRI_TRAFFIC.get(args.workload) if args.scale == 1.0 else None,
                "algo_bytes_per_edge": ALGO_BYTES["tri"], "kernel_ms": ph["tri"],
                "phases": {k: {"ms": round(ph[k], 4), "algo_GBps": round(gbs(k), 1),
                               "frac": round(gbs(k) / peak, 4)} for k in ph if ph[k] > 0}}

    # count only (graph resident)
    count_ms = None
    g = tm.build_async(src, dst, tt, stream) if not args.no_count_only else None
    torch.cuda.synchronize()
    if g is not None:
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
    out_cells = cells.cpu().numpy()
    _, bad = tm.merge(out_cells)

    e2e = None
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
            out = tm.count(g, delta)
            g.free()
            times.append(time.perf_counter() - st)
        e2e_step = sum(times) / len(times)
        if dist:
            x = torch.tensor([e2e_step], device="cuda", dtype=torch.float64)
            dist.all_reduce(x, op=dist.ReduceOp.MAX)
            e2e_step = float(x.item())
        e2e = {"value": world * m / e2e_step, "unit": UNIT, "h2d_bytes_per_step": 16 * m,
               "d2h_bytes_per_step": 36 * 8, "ms_per_step": e2e_step * 1e3}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, d, t, delta, args.cpu_sample_days)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded generators standing in for the paper's SNAP datasets)",
            "config": {"workload": wl["desc"], "m": m, "delta": delta, "scale": args.scale,
                       "l2": "inputs (16 B/edge) larger than the 129 MB L2; no flush",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": launches,
            "count_only": ({"value": m / (count_ms / 1e3), "unit": UNIT, "ms": count_ms}
                           if count_ms else None),
            "phases_ms": {k: round(v, 4) for k, v in ph.items()},
            "isomorphism_mismatches": bad,
        }))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
