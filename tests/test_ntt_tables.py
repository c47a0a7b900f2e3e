"""The transform product's constants (host code, csrc/ntt_tables.h) checked on
the CPU: primes, orders of the roots of unity, Shoup companions, Montgomery,
scaling and Garner constants, the three-prime bound, and exact products
through the tables against the schoolbook product (tests/ntt_check.cpp)."""

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_06386_gb300", "csrc")


def test_ntt_tables(tmp_path):
    exe = str(tmp_path / "ntt_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "ntt_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
