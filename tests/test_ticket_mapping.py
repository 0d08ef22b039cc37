"""The fused loops' index arithmetic on the CPU, compiled from the library's
own headers with nvcc as host code: the ticket -> (frame, tile) mapping
(tc_ticket_tile) and the ring slots taken from a per-launch base
(RingSlot)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1802_06625_b300", "csrc")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_ticket_mapping_is_a_bijection_onto_frames_and_tiles(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = tmp_path / "ticket_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(HERE, "..", "include"),
                    "-DPRUNE_BUILD", os.path.join(HERE, "native", "ticket_check.cu"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split().count("ok") == 2, r.stdout


def test_ring_slot_equals_the_modulo(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = tmp_path / "ring_slot_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-I", CSRC, "-I",
                    os.path.join(HERE, "..", "include"), "-DPRUNE_BUILD", os.path.join(HERE, "native", "ring_slot_check.cu"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok"), r.stdout
