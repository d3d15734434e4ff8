"""Host logic of the serving loop without a GPU: the output arena (first fit,
coalescing, shrinking, peak accounting) and the admission rule (arrival order;
only requests that need no output memory may pass a head that waits for it),
compiled from the library's own header with the host C++ compiler."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_and_admission(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "serve_arena_test"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2408_11971_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "serve_arena_test.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "ok" in r.stdout
