"""The integer-unit float operations of csrc/sor_bits.cuh (exact widening,
exact times 4, round-to-nearest-even narrowing), compiled for the host with
nvcc and compared bit for bit with the host's IEEE arithmetic on random bit
patterns of every class and on boundary values."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1401_0763_gb300", "csrc")


def test_bit_operations_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "bits_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe, os.path.join(HERE, "bits_check.cu")],
                   check=True, capture_output=True)
    r = subprocess.run([exe, "400000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "widen 0 times4 0 narrow 0" in r.stdout
