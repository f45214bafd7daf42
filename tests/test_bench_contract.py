"""bench.py's JSON line on the GPU (a small workload, so the test is quick): every key of the
benchmark contract, the roofline and CPU-baseline objects, and consistent numbers."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_bench_json_line_on_a_small_workload():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "C3:24", "--steps", "5",
                          "--warmup", "3", "--no-serve", "--sample-fraction", "0.25"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3 and d["dtype"] == "f64"
    assert d["value"] > 0 and abs(d["value"] - d["config"]["elements"] / (d["ms_per_step"] * 1e6)) < 1e-6 * d["value"]
    roof = d["roofline"]
    assert roof["bound"] in ("alu", "hbm") and 0 < roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    e2e = d["e2e"]
    assert e2e["h2d_bytes_per_step"] == 8 * d["config"]["dofs"]
    assert e2e["d2h_bytes_per_step"] == 8 * d["config"]["dofs"] + 8
    if "l2" in e2e:
        # inputs that fit in L2: value evicts L2 before every step, the host-buffer steps run
        # back to back, so the two are not comparable
        assert e2e["value"] > 0 and "l2" in d["config"]
    else:
        assert 0 < e2e["value"] <= d["value"] * 1.05
    assert d["gpu_launches"] == 3 * d["steps"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert set(d["variants"]) >= {"df64", "f32", "f64_hessian_vector"}
