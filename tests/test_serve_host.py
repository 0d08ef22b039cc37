"""Host logic of the request loop on the CPU: the device-memory arena
(first-fit with coalescing), the per-stream layout and the step planner
(admission order, frames per step, result-FIFO backpressure, delay-token
chaining), compiled from the library's own header with g++."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1802_06625_b300", "csrc")


def test_serve_host_logic(tmp_path):
    exe = tmp_path / "serve_host_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-I", CSRC, os.path.join(HERE, "native", "serve_host_check.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split().count("ok") == 3, r.stdout
