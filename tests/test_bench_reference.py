"""bench.py's reference arm (the CPU oracle on the benchmark workload) on the host: one JSON line
with the keys the benchmark contract names, a positive rate measured on the configured steps, and
only rank 0 working under a multi-rank launch."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    res = run_bench(None, "--steps", "3", "--warmup", "3")
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "syndromes/sec" and d["unit"] == "syndromes/s"
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["ms_per_step"] > 0 and d["data"] == "synthetic" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["shots"] > 0 and st["shots_per_s"] > 0
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["p999_us"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    res = run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "3", "--warmup", "3",
                    "--gpus", "2")
    assert res.returncode == 0, res.stderr[-2000:]
    assert not [l for l in res.stdout.splitlines() if l.startswith("{")]
