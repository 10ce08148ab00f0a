"""bench.py end to end on the small training-step workload (100,000 pairs, m = 150, n = 300):
the device-timed step, the two end-to-end paths (host pipeline and the device API with pinned
copies) and the roofline object all run and yield one well-formed JSON line.  The numbers
themselves are not checked here (a test run shares the GPU with nothing but is short)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _last_json(text):
    for line in reversed(text.strip().splitlines()):
        line = line.strip()
        if line.startswith("{"):
            return json.loads(line)
    raise AssertionError("no JSON line:\n" + text[-2000:])


def test_bench_line_on_the_small_training_step():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = subprocess.run([sys.executable, "bench.py", "--workload", "c3_grad", "--steps", "1",
                        "--warmup", "3", "--no-cpu-baseline"], cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    j = _last_json(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "roofline", "e2e",
              "gpu_launches", "clocks"):
        assert k in j, k
    assert j["value"] > 0 and j["ms_per_step"] > 0 and j["gpu_launches"] > 0
    assert j["e2e"]["value"] > 0
    assert j["e2e"]["h2d_bytes_per_step"] > 0 and j["e2e"]["d2h_bytes_per_step"] > 0
    ro = j["roofline"]
    assert ro["bound"] == "alu" and 0 < ro["frac"] < 1.5
    assert abs(ro["frac"] - ro["achieved"] / ro["peak"]) < 1e-9
