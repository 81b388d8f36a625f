"""The auxiliary kernels' node coordinates (node_xy, NodeWalk of
node_xy.cuh), compiled for the host and checked against 64-bit division:
sampled indices on both sides of 2^31 for many lattice widths, and every
node of grid-stride walks of the drift kernels' strides
(tests/native/node_xy_check.cu)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_node_xy_host_check(tmp_path):
    nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "node_xy_check")
    src = os.path.join(HERE, "native", "node_xy_check.cu")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:]
