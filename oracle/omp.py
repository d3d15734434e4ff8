"""CPU throughput baseline: the oracle's codec and operators with an OpenMP loop
over blocks (``hoszp_omp.c``, which includes the oracle's source), the
organisation of the paper's CPU design (Sec. VI-A). BENCHMARK AND TEST
INFRASTRUCTURE ONLY: ``bench.py`` times it on every host core next to the
single-threaded oracle, and the tests check its output against the oracle's.
Mean and variance are finished from the exact sums as the oracle does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

from . import OracleError, _check, _ptr, _stream, bound, header

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hoszp_omp.c")
_DEP = os.path.join(_HERE, "hoszp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hoszp_omp.c (with the oracle's source) into liboracle_omp.so."""
    with _lock:
        stale = not os.path.exists(_LIB) or any(
            os.path.getmtime(_LIB) < os.path.getmtime(p) for p in (_SRC, _DEP))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC",
                 "-fopenmp", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P, U64, SZ, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
    D = ctypes.c_double
    lib.omp_compress.argtypes = [P, U64, P, I, D, I, P, SZ, P]
    lib.omp_decompress.argtypes = [P, SZ, P, U64]
    lib.omp_negate.argtypes = [P, SZ, P, SZ, P]
    lib.omp_add_scalar.argtypes = [P, SZ, D, P, SZ, P]
    lib.omp_mul_scalar.argtypes = [P, SZ, D, P, SZ, P]
    lib.omp_add.argtypes = [P, SZ, P, SZ, P, SZ, P]
    lib.omp_sums.argtypes = [P, SZ, P, P, P, P, P, P]
    for f in (lib.omp_compress, lib.omp_decompress, lib.omp_negate, lib.omp_add_scalar,
              lib.omp_mul_scalar, lib.omp_add, lib.omp_sums, lib.omp_threads):
        f.restype = I
    _lib = lib
    return lib


def threads() -> int:
    """OpenMP threads a parallel loop uses (OMP_NUM_THREADS, else every core)."""
    return int(_load().omp_threads())


def compress(x, dims=None, eb: float = 1e-3, mode: str = "abs") -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = tuple(x.shape) if dims is None else tuple(dims)
    d = np.array(list(dims) + [0] * (3 - len(dims)), np.uint32)
    cap = bound(x.size)
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(_load().omp_compress(_ptr(x), x.size, _ptr(d), len(dims), float(eb),
                                1 if mode == "rel" else 0, _ptr(out), cap, _ptr(nbytes)),
           "omp_compress")
    return out[: int(nbytes[0])].copy()


def decompress(c) -> np.ndarray:
    c = _stream(c)
    n = header(c)["n"]
    x = np.zeros(n, np.float32)
    _check(_load().omp_decompress(_ptr(c), c.size, _ptr(x), n), "omp_decompress")
    return x


def _unary(fn, c, *args) -> np.ndarray:
    c = _stream(c)
    cap = bound(header(c)["n"])
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(fn(_ptr(c), c.size, *args, _ptr(out), cap, _ptr(nbytes)), fn.__name__)
    return out[: int(nbytes[0])].copy()


def negate(c) -> np.ndarray:
    return _unary(_load().omp_negate, c)


def add_scalar(c, s: float) -> np.ndarray:
    return _unary(_load().omp_add_scalar, c, ctypes.c_double(s))


def mul_scalar(c, s: float) -> np.ndarray:
    return _unary(_load().omp_mul_scalar, c, ctypes.c_double(s))


def add(a, b) -> np.ndarray:
    a, b = _stream(a), _stream(b)
    cap = bound(header(a)["n"])
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(_load().omp_add(_ptr(a), a.size, _ptr(b), b.size, _ptr(out), cap, _ptr(nbytes)),
           "omp_add")
    return out[: int(nbytes[0])].copy()


def sums(c):
    c = _stream(c)
    s1h = np.zeros(1, np.int64)
    s1l, s2h, s2l, n = (np.zeros(1, np.uint64) for _ in range(4))
    e = np.zeros(1, np.float32)
    _check(_load().omp_sums(_ptr(c), c.size, _ptr(s1h), _ptr(s1l), _ptr(s2h), _ptr(s2l), _ptr(n),
                            _ptr(e)), "omp_sums")
    s1 = (int(s1h[0]) << 64) | int(s1l[0])
    return s1, (int(s2h[0]) << 64) | int(s2l[0]), int(n[0]), e[0]


def mean(c) -> float:
    s1, _, n, e = sums(c)
    if n == 0:
        raise OracleError(-1, "omp_mean")
    return float(Fraction(s1, n) * 2 * Fraction(float(e)))


def var(c) -> float:
    s1, s2, n, e = sums(c)
    if n == 0:
        raise OracleError(-1, "omp_var")
    a = 2 * Fraction(float(e))
    return float(a * a * Fraction(n * s2 - s1 * s1, n * n))
