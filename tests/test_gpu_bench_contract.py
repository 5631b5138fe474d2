"""GPU: bench.py prints the one JSON line the measurement contract asks for.

A short run (5 timed steps of the 2048 x 2048 x 5 workload) through the same entry point
the round-end measurement uses; checks every key, the units and the internal arithmetic
(value = sites x N / time per step, roofline fraction = achieved / peak, launches = 2 per
step), not the speed."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "5", "--warmup", "3",
           "--no-variants", "--no-cpu-baseline"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] >= 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["config"]["workload"] == "n5_2048x2048" and d["dtype"] == "f32"
    sites_n = 2048 * 2048 * 5
    assert abs(d["value"] - sites_n / (d["ms_per_step"] * 1e-3) / 1e6) < 1e-6 * d["value"]
    rl = d["roofline"]
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert abs(rl["frac"] - rl["achieved"] / rl["peak"]) < 1e-9
    assert abs(rl["achieved"] - 72 * sites_n / (d["ms_per_step"] * 1e-3) / 1e9) < 1e-6 * rl["achieved"]
    e2e = d["e2e"]
    assert e2e["unit"] == d["unit"] and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert e2e["job_steps"] == 2000
    assert abs(e2e["h2d_bytes_per_step"] - (5 + 2) * 2048 * 2048 * 8 / 2000) < 1e-6 * e2e["h2d_bytes_per_step"]
    assert d["gpu_launches"] == 2 * d["steps"]
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    assert d["clocks"]["samples"] > 0 and d["clocks"]["sm_mhz"] > 0
