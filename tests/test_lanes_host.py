"""The two-lanes-per-block decode of the variance and the covariance
(hz_lanes.cuh) against brute force on the host: the header is
host-compilable, the device intrinsics running as its host definitions.
Every rate 0..31, short last blocks, signs on zero magnitudes, ignored bits
at position 0, both accumulation widths; the exact sums S1 and S2 of single
blocks and sum q_A q_B, sum q_A, sum q_B of block pairs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_lanes_decode_sums(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "lanes_decode_test"
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-Wno-unknown-pragmas",
                    "-I", os.path.join(ROOT, "paper_2408_11971_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "lanes_decode_test.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout
