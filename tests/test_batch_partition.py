"""The batched tensor-core FIR's per-CTA work split (contiguous shares of
equal estimated cost) on the CPU, compiled from the library's own header
with g++."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1802_06625_b300", "csrc")


def test_fir_cost_partition(tmp_path):
    exe = tmp_path / "batch_partition_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-I", CSRC,
                    os.path.join(HERE, "native", "batch_partition_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split().count("ok") == 3, r.stdout
