"""Host check of the library's integer-pipe binary32 <-> binary64 conversions
(csrc/cvt.cuh, __host__ __device__): compiled with the host C++ compiler and
compared bit for bit with the host's IEEE 754 conversions - the widening for
every binary32 value, the round-to-nearest-even narrowing for seeded random
binary64 values, rounding midpoints and range boundaries."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "cvt_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "native", "cvt_check.cpp")], check=True)
    r = subprocess.run([exe, "5000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().startswith("ok"), r.stdout
