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


def test_reference_config_is_the_gpu_arms():
    """Both arms describe the workload with the same config (the GPU arm
    calls config_of on the workload's jobs)."""
    bench = bench_module()
    d = json.loads(run()[0])
    assert d["config"] == bench.config_of("plain_481x321", bench.workload_jobs("plain_481x321"))


def test_oracle_sample_of_the_4k_batch():
    """Images above 1920x1080 are timed by their top-left quarter with a
    quarter of the superpixels; smaller ones as they are."""
    import numpy as np
    from paper_1309_3848_gb300 import synth
    bench = bench_module()
    jobs = synth.batch_4k(2) + synth.plain_481()
    imgs = [np.zeros((j.image.height, j.image.width, 3), np.uint8) for j in jobs]
    imgs[0][:1080, :1920] = 7
    sj, si, what = bench.oracle_sample(jobs, imgs)
    assert [(j.image.width, j.image.height, j.num_superpixels) for j in sj] == \
        [(1920, 1080, 1250), (1920, 1080, 1250), (481, 321, 200)]
    assert all(j.bins_per_channel == o.bins_per_channel and j.levels == o.levels and
               j.iters_per_level == o.iters_per_level for j, o in zip(sj, jobs))
    assert si[0].shape == (1080, 1920, 3) and int(si[0].min()) == 7 and si[2] is imgs[2]
    assert "quarter" in what
