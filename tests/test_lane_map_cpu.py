"""The step kernels' work mapping (make_geom, lane_pos of d2q9_pull.cuh),
compiled for the host and checked exhaustively on tiny lattices: every real
chunk is covered exactly once, padding slots are inactive, the neighbour
flags are right, tasks start on 128-byte lines, and the multiply-shift row
division is exact (tests/native/lane_map_check.cu)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_lane_map_host_check(tmp_path):
    nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "lane_map_check")
    src = os.path.join(HERE, "native", "lane_map_check.cu")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:]
