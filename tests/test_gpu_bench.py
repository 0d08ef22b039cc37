"""The bench line's contract on the GPU: a short run of bench.py (48 frames
of the plain-large graph, one CPU-baseline frame) prints one JSON line with
every key the contract asks for, the roofline against the measured peak and
the end-to-end leg through the host."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")


def test_bench_line_contract():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cmd = [sys.executable, "bench.py", "--steps", "1", "--warmup", "3", "--frames", "48", "--C", "48",
           "--no-batched", "--no-serving", "--no-dpd", "--no-small", "--no-diff", "--e2e-frames", "3", "--cpu-frames", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("plain_F4096_B1024_T64_N32")
    roof = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["bound"] == "hbm" and 0 < roof["frac"] < 1.2 and roof["kernel"] == "firing_loop_ws_kernel"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 3 * 4096 * 1024 * 8 and e["d2h_bytes_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and cb["sample"]
    assert d["gpu_launches"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
