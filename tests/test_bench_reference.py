"""bench.py's reference arm (the oracle on the host cores) on the CPU: one
JSON line with the bench's metric, the oracle as its CPU baseline and no
host-device traffic; ranks other than 0 print nothing."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_module():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def run(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "plain_481x321", "--steps", "1",
           "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    return [line for line in res.stdout.splitlines() if line.strip()]


def test_reference_line():
    lines = run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    bench = bench_module()
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Mpixel/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "plain_481x321" and d["config"]["pixels_per_step"] == 481 * 321
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_other_ranks_print_nothing():
    assert run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
