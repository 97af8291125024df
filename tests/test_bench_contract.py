"""The bench's one-line JSON result: the keys and types the benchmark
contract asks for, on the reference arm (CPU, the oracle) and on a short
default run (GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e"}


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "2", "--warmup", "3"], timeout=600)
    assert BASE_KEYS <= set(d) and d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["config"]["workload"] == "kolmogorov_d3q27_512cubed"
    assert d["config"]["nodes_per_step"] == 512 ** 3 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "512 x 64 x 64" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_default_run_line():
    d = _run(["--steps", "4", "--warmup", "3", "--no-cpu-baseline", "--no-extras"], timeout=900)
    assert BASE_KEYS <= set(d) and "impl" not in d
    assert d["steps"] == 4 and d["warmup"] == 3 and d["value"] > 0 and d["dtype"] == "f64"
    assert d["config"]["workload"] == "kolmogorov_d3q27_512cubed" and "l2" in d["config"]
    r = d["roofline"]
    assert r["bound"] == "alu" and r["peak"] > 0 and r["achieved"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-12 * r["frac"]
    assert "traffic" in r and "hbm" in r and "flops" in r and r["ops_per_node"] == 254
    p = d["fp64_peak"]
    assert p["sm_count"] == d["device"]["sm_count"] > 0 and p["fma_ginst_per_s"] > 0 and p["add_ginst_per_s"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == "MLUPS" and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == d["steps"]  # one batched launch per step
    c = d["clocks"]
    assert c["sm_mhz"] > 0 and c["sm_max_mhz"] > 0 and isinstance(c["reasons"], list)
