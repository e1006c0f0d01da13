"""The main arm of bench.py prints one JSON line with the contract's keys
(small workload, no CPU leg): the metric and its value, the end-to-end
number with the bytes copied each step, the launch count, the roofline of
the dominant kernel and the clocks seen during the timed steps."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_main_arm_json_contract():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "uniform4k",
                          "--steps", "3", "--warmup", "3", "--no-cpu-baseline", "--no-extras"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "gpu_launches", "roofline", "clocks"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] >= 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "uniform4k"
    n = line["config"]["n"]
    e = line["e2e"]
    assert e["value"] > 0 and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 16 * n and e["d2h_bytes_per_step"] == 16 * n + 8
    # every step launches the same kernels: at least one per stage (bin, sort,
    # near field, replacement, contraction, far field at the charges, unsplit)
    assert line["gpu_launches"] % line["steps"] == 0
    assert line["gpu_launches"] >= 8 * line["steps"]
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] in ("hbm", "tensor", "alu") and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 * max(1.0, r["frac"])
