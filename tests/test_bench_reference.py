"""The benchmark's reference arm, the oracle on the host cores, on the CPU.

A single process prints one JSON line of the benchmark contract, with the
oracle described as the CPU baseline and an end-to-end object without device
copies. A rank other than 0 of a multi-process launch prints nothing and
exits 0.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env=None):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=600, cwd=ROOT,
                          env=env if env is not None else dict(os.environ))


ARGS = ["--impl", "reference", "--workload", "tiny", "--steps", "2", "--warmup", "1"]


def test_reference_arm_prints_the_contract_line():
    r = run_bench(ARGS)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "edges/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["m"] == 20000 and line["config"]["delta"] == 3600
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == line["value"] and cb["unit"] == line["unit"]
    e = line["e2e"]
    assert e["value"] == line["value"] and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = run_bench(ARGS + ["--gpus", "2"], env=env)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
