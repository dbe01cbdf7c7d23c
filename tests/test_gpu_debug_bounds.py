"""The bounds-checked debug build (every histogram, size, bin, label and
decision index checked on the device; a trip sets the error word and reads
as SEEDS_ERR_DEVICE) runs edge sizes, random jobs, every tuning shape, LAB,
means iterations and an anytime stop without a trip, with the oracle's
labels."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def debug_lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1309_3848_gb300 import _build
    return _build.build_debug()


def test_no_bounds_trip_and_oracle_labels(debug_lib):
    env = dict(os.environ, SEEDS_LIB=debug_lib)
    res = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_run.py")], env=env,
                         capture_output=True, text=True, timeout=1200)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["images"] > 20
    for tuning, bad in out["mismatches"].items():
        assert not bad, "tuning %s: %s" % (tuning, bad[:3])
