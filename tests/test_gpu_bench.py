"""bench.py itself on a small case: it runs, prints one JSON line with the keys
the measurement contract asks for, and its CPU baseline agrees with the GPU."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=900):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_bench_window_line():
    d = _bench("--steps", "2", "--warmup", "1", "--width", "20000", "--no-extras")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "roofline",
              "e2e", "clocks", "gpu_launches", "cpu_baseline", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["gpu_launches"] > 0 and d["config"]["congruences"] == "BB2244+EE2004"
    r = d["roofline"]
    assert r["bound"] == "alu" and r["kernel"] == "accumulate_m31" and r["terms_per_clk_sm"] > 0
    assert r["traffic"] is None  # a partial window: no full-launch traffic figure
    assert d["cpu_baseline"]["agrees_with_gpu"] and d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert d["e2e"]["h2d_bytes_per_step"] == 8 * d["config"]["primes_per_gpu"]


def test_bench_top_line():
    d = _bench("--workload", "top", "--steps", "1", "--warmup", "1", "--width", "400", "--no-extras")
    assert d["roofline"]["kernel"] == "accumulate_m64" and d["value"] > 0
    assert d["config"]["congruences"] == "BB3802+EE4122" and d["hits"] == 0
