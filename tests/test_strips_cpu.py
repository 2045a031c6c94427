"""The strip tables of the data-flow kernels (csrc/sor_strips.cuh), compiled
for the host with nvcc: coverage of every interior row and column tile
exactly once, the numbering the kernels decode, accesses inside the arrays,
and neighbour lists that contain every strip the 7-point (cube) and 9-point
stencils reach, checked by brute force over many sizes and warp counts."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1401_0763_gb300", "csrc")


def test_strip_tables_and_neighbours(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "strips_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe, os.path.join(HERE, "strips_check.cu")],
                   check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "strips: 0 failures" in r.stdout
