"""The slot ranges of the batched step's constant-memory tables
(SlotRanges of csrc/slots.h), compiled for the host: first fit, release
and reuse, exhaustion and bad sizes, and random reserve / release
sequences against a brute-force occupancy model
(tests/native/slots_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_slot_ranges_host_check(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "slots_check")
    src = os.path.join(HERE, "native", "slots_check.cpp")
    subprocess.run([cxx, "-O2", "-std=c++17", "-Wall", src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:]
