"""The C ABI library builds for sm_103a, loads, and exports every function that
include/hoszp.h declares (no GPU needed: nothing is launched)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hoszp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hoszp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_11971_gb300 import build

    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["hoszp_compress", "hoszp_decompress", "hoszp_negate", "hoszp_add_scalar",
              "hoszp_mul_scalar", "hoszp_add", "hoszp_mean", "hoszp_var", "hoszp_ctx_create",
              "hoszp_ctx_destroy", "hoszp_get_status", "hoszp_compress_bound"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hoszp_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    handle = ctypes.CDLL(lib)
    for f in declared_functions():
        assert getattr(handle, f) is not None


def test_compress_bound_and_host_checks(lib):
    import paper_2408_11971_gb300 as hz

    assert hz.compress_bound(0) == 64
    n = 1000
    nb = (n + 63) // 64
    assert hz.compress_bound(n) == 64 + (nb + 15) // 16 * 16 + (4 * nb + 15) // 16 * 16 + 8 * nb * 32
    L = hz.load_library()
    # argument errors are returned before anything touches a device
    assert L.hoszp_ctx_create(None, 0) == -1
    assert L.hoszp_compress(None, None, 0, None, 1, 1.0, 0, None, 0, None, None) == -1
    assert L.hoszp_mean(None, None, 0, None, None) == -1
    # the operators beyond the step: null context or buffers are argument errors
    assert L.hoszp_sub_scalar(None, None, 0, 1.0, None, 0, None, None) == -1
    assert L.hoszp_mul_scalar_exact(None, None, 0, 1.0, None, 0, None, None) == -1
    assert L.hoszp_std(None, None, 0, None, None) == -1
    assert L.hoszp_block_means(None, None, 0, None, 0, None) == -1
    assert L.hoszp_cov(None, None, 0, None, 0, None, None) == -1
    assert L.hoszp_hadamard(None, None, 0, None, 0, None, 0, None, 0, None, None) == -1
    assert L.hoszp_batch_decompress(None, None, None) == -1
    assert L.hoszp_finish_sums(None, None, ctypes.c_float(1.0), None, None, None) == -1
    assert L.hoszp_concat(None, 0, None, None, None, 1, None, 0, None, None) == -1
    assert L.hoszp_selftest_wait(None, 0, 1, None) == -1


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    from paper_2408_11971_gb300 import _binding

    monkeypatch.setattr(_binding, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_binding, "_lib", None)
    with pytest.raises(RuntimeError):
        _binding.load_library()
