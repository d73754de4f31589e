"""bench.py's output contract on a small case: one JSON line with the keys the harness
reads, the roofline and end-to-end objects, the launch count and the clock samples."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_bench_line_contract():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--headline-batch", "100000", "--steps", "3",
           "--warmup", "3", "--e2e-steps", "3", "--no-path-stage", "--no-serve", "--no-paper-generator",
           "--no-curation", "--no-topology", "--no-cpu-baseline", "--no-other-configs", "--no-two-stage"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert "workload" in d["config"]
    roof = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["bound"] in ("hbm", "alu", "tensor") and 0 < roof["frac"] < 2
    assert abs(roof["achieved"] / roof["peak"] - roof["frac"]) < 1e-6
    e2e = d["e2e"]
    assert e2e["unit"] == d["unit"] and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0


@pytest.mark.parametrize("nmax", [8, 20])
def test_bench_profiling_mode(nmax):
    """bench.py --profile-kernels (the launches the committed ncu summaries capture) runs
    to completion on a small case."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--profile-kernels", "--batch", "20000",
           "--profile-nmax", str(nmax)]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert d["profile_kernels"] == "done" and d["n_max"] == nmax and d["valid_rows"] > 0
