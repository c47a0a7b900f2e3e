"""The serving loop's ring allocator (host code, csrc/serve_ring.h) checked on
the CPU against a model of the live ranges: randomised allocation and
out-of-order release, exhaustion and recovery (tests/ring_check.cpp)."""

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_06386_gb300", "csrc")


def test_ring_allocator(tmp_path):
    exe = str(tmp_path / "ring_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "ring_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
