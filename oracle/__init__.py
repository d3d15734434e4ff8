"""CPU oracle for the HoSZp codec and homomorphic operators (arXiv 2408.11971).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``. The library never imports it.

The arithmetic lives in ``hoszp_oracle.c`` (plain single-threaded C, compiled
with ``-O2 -ffp-contract=off``); this module compiles it on first use, loads it
with ctypes and finishes the reductions exactly with Python integers and
fractions:

* mean (Sec. V-B): the exact rational ``S1 / n * 2 eps_q`` rounded once to double;
* variance (Sec. V-B): the exact rational ``(2 eps_q)^2 (n S2 - S1^2) / n^2``
  (population variance of the quantized integers) rounded once to double.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hoszp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# error codes of the oracle (same numbering as the library ABI)
CODES = {
    0: "OK", -1: "ARG", -2: "CAPACITY", -3: "FORMAT", -4: "MISMATCH",
    -5: "RANGE", -6: "OVERFLOW", -7: "NONFINITE",
}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {CODES.get(code, code)} ({code})")
        self.code = code
        self.name = CODES.get(code, str(code))


def build(force: bool = False) -> str:
    """Compile hoszp_oracle.c into liboracle.so next to it (gcc, no OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC",
                 "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    U64 = ctypes.c_uint64
    SZ = ctypes.c_size_t
    I = ctypes.c_int
    lib.orc_bound.restype = SZ
    lib.orc_bound.argtypes = [U64]
    lib.orc_compress.argtypes = [P, U64, P, I, ctypes.c_double, I, P, SZ, P]
    lib.orc_decompress.argtypes = [P, SZ, P, U64]
    lib.orc_decode_q.argtypes = [P, SZ, P, U64]
    lib.orc_negate.argtypes = [P, SZ, P, SZ, P]
    lib.orc_add_scalar.argtypes = [P, SZ, ctypes.c_double, P, SZ, P]
    lib.orc_mul_scalar.argtypes = [P, SZ, ctypes.c_double, P, SZ, P]
    lib.orc_add.argtypes = [P, SZ, P, SZ, P, SZ, P]
    lib.orc_concat.argtypes = [ctypes.c_uint32, P, P, P, I, P, SZ, P]
    lib.orc_sub.argtypes = [P, SZ, P, SZ, P, SZ, P]
    lib.orc_sums.argtypes = [P, SZ, P, P, P, P, P, P]
    lib.orc_sub_scalar.argtypes = [P, SZ, ctypes.c_double, P, SZ, P]
    lib.orc_mul_scalar_exact.argtypes = [P, SZ, ctypes.c_double, P, SZ, P]
    lib.orc_hadamard.argtypes = [P, SZ, P, SZ, P, SZ, P]
    lib.orc_block_means.argtypes = [P, SZ, P, U64]
    lib.orc_cov_sums.argtypes = [P, SZ, P, SZ, P, P, P, P, P, P, P]
    lib.orc_header.argtypes = [P, SZ, P, P, P, P, P, P]
    lib.orc_eps_q.argtypes = [ctypes.c_double, P]
    lib.orc_quantize.argtypes = [ctypes.c_float, ctypes.c_float, P]
    lib.orc_quantize_scalar.argtypes = [ctypes.c_double, ctypes.c_float, P]
    lib.orc_dequantize.restype = ctypes.c_float
    lib.orc_dequantize.argtypes = [ctypes.c_int64, ctypes.c_float]
    lib.orc_mul_requant.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_float, P]
    for f in (lib.orc_compress, lib.orc_decompress, lib.orc_decode_q, lib.orc_negate,
              lib.orc_add_scalar, lib.orc_mul_scalar, lib.orc_add, lib.orc_sums,
              lib.orc_header, lib.orc_eps_q, lib.orc_quantize, lib.orc_quantize_scalar,
              lib.orc_mul_requant, lib.orc_concat):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(rc, what)


def _stream(c) -> np.ndarray:
    return np.ascontiguousarray(np.frombuffer(bytes(c), dtype=np.uint8)) if not isinstance(
        c, np.ndarray) else np.ascontiguousarray(c, dtype=np.uint8)


def bound(n: int) -> int:
    return int(_load().orc_bound(n))


def eps_q(eps: float) -> np.float32:
    out = np.zeros(1, np.float32)
    _check(_load().orc_eps_q(float(eps), _ptr(out)), "eps_q")
    return out[0]


def quantize(x: float, e_q) -> int:
    out = np.zeros(1, np.int64)
    _check(_load().orc_quantize(float(np.float32(x)), float(np.float32(e_q)), _ptr(out)),
           "quantize")
    return int(out[0])


def quantize_scalar(s: float, e_q) -> int:
    out = np.zeros(1, np.int64)
    _check(_load().orc_quantize_scalar(float(s), float(np.float32(e_q)), _ptr(out)),
           "quantize_scalar")
    return int(out[0])


def dequantize(q: int, e_q) -> np.float32:
    return np.float32(_load().orc_dequantize(int(q), float(np.float32(e_q))))


def mul_requant(q: int, rho: int, e_q) -> int:
    out = np.zeros(1, np.int64)
    _check(_load().orc_mul_requant(int(q), int(rho), float(np.float32(e_q)), _ptr(out)),
           "mul_requant")
    return int(out[0])


def compress(x, dims=None, eb: float = 1e-3, mode: str = "abs") -> np.ndarray:
    """Compress float32 values; dims defaults to the array's shape (1..3 dims)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if dims is None:
        dims = x.shape if x.ndim >= 1 else (x.size,)
    dims = tuple(int(d) for d in dims)
    d3 = np.zeros(3, np.uint32)
    d3[: len(dims)] = dims
    n = x.size
    cap = bound(n)
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    flat = x.reshape(-1)
    rc = _load().orc_compress(_ptr(flat), n, _ptr(d3), len(dims), float(eb),
                              1 if mode == "rel" else 0, _ptr(out), cap, _ptr(nbytes))
    _check(rc, "compress")
    return out[: int(nbytes[0])].copy()


def header(c) -> dict:
    c = _stream(c)
    v = [np.zeros(1, t) for t in (np.uint64, np.uint64, np.uint64, np.uint32, np.float32,
                                  np.uint64)]
    _check(_load().orc_header(_ptr(c), c.size, *[_ptr(a) for a in v]), "header")
    return dict(n=int(v[0][0]), nnc=int(v[1][0]), R=int(v[2][0]), qbound=int(v[3][0]),
                eps_q=v[4][0], size=int(v[5][0]))


def decode_q(c) -> np.ndarray:
    c = _stream(c)
    n = header(c)["n"]
    q = np.zeros(max(n, 1), np.int64)
    _check(_load().orc_decode_q(_ptr(c), c.size, _ptr(q), n), "decode_q")
    return q[:n]


def decompress(c) -> np.ndarray:
    c = _stream(c)
    n = header(c)["n"]
    x = np.zeros(max(n, 1), np.float32)
    _check(_load().orc_decompress(_ptr(c), c.size, _ptr(x), n), "decompress")
    return x[:n]


def _unary(fn, c, *args) -> np.ndarray:
    c = _stream(c)
    cap = bound(header(c)["n"])
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(fn(_ptr(c), c.size, *args, _ptr(out), cap, _ptr(nbytes)), fn.__name__)
    return out[: int(nbytes[0])].copy()


def negate(c) -> np.ndarray:
    return _unary(_load().orc_negate, c)


def add_scalar(c, s: float) -> np.ndarray:
    return _unary(_load().orc_add_scalar, c, ctypes.c_double(s))


def sub_scalar(c, s: float) -> np.ndarray:
    """Scalar subtraction (Sec. V-A): O' = O - rho_s, rho_s = Eq. 3 of s."""
    return _unary(_load().orc_sub_scalar, c, ctypes.c_double(s))


def mul_scalar(c, s: float) -> np.ndarray:
    return _unary(_load().orc_mul_scalar, c, ctypes.c_double(s))


def mul_scalar_exact(c, s: float) -> np.ndarray:
    """Multiplication by the scalar itself: q' = floor(q s + 1/2), exactly."""
    return _unary(_load().orc_mul_scalar_exact, c, ctypes.c_double(s))


def add(a, b) -> np.ndarray:
    a = _stream(a)
    b = _stream(b)
    cap = bound(header(a)["n"])
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(_load().orc_add(_ptr(a), a.size, _ptr(b), b.size, _ptr(out), cap, _ptr(nbytes)),
           "add")
    return out[: int(nbytes[0])].copy()


def concat(streams, dims) -> np.ndarray:
    """Streams of consecutive shards of one field (same bound; every shard but
    the last of whole blocks) joined into the field's stream of shape dims."""
    ss = [_stream(c) for c in streams]
    k = len(ss)
    ptrs = (ctypes.c_void_p * k)(*[c.ctypes.data for c in ss])
    sizes = (ctypes.c_size_t * k)(*[c.size for c in ss])
    d = (ctypes.c_uint32 * 3)(*(list(dims) + [0, 0, 0])[:3])
    n = int(np.prod(dims))
    cap = bound(n)
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(_load().orc_concat(k, ptrs, sizes, d, len(dims), _ptr(out), cap, _ptr(nbytes)),
           "concat")
    return out[: int(nbytes[0])].copy()


def hadamard(a, b) -> np.ndarray:
    """Hadamard product (Sec. V-C): q' = floor(2 eps q_A q_B + 1/2), re-encoded."""
    a = _stream(a)
    b = _stream(b)
    cap = bound(header(a)["n"])
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(_load().orc_hadamard(_ptr(a), a.size, _ptr(b), b.size, _ptr(out), cap, _ptr(nbytes)),
           "hadamard")
    return out[: int(nbytes[0])].copy()


def sub(a, b) -> np.ndarray:
    """Element-wise subtraction A - B (Sec. V-C): q' = q_A - q_B, re-encoded."""
    a = _stream(a)
    b = _stream(b)
    cap = bound(header(a)["n"])
    out = np.zeros(cap, np.uint8)
    nbytes = np.zeros(1, np.uint64)
    _check(_load().orc_sub(_ptr(a), a.size, _ptr(b), b.size, _ptr(out), cap, _ptr(nbytes)),
           "sub")
    return out[: int(nbytes[0])].copy()


def sums(c):
    """Exact (S1, S2, n, eps_q): S1 = sum q, S2 = sum q^2 over the stream."""
    c = _stream(c)
    s1h = np.zeros(1, np.int64)
    s1l, s2h, s2l, n = (np.zeros(1, np.uint64) for _ in range(4))
    e = np.zeros(1, np.float32)
    _check(_load().orc_sums(_ptr(c), c.size, _ptr(s1h), _ptr(s1l), _ptr(s2h), _ptr(s2l),
                            _ptr(n), _ptr(e)), "sums")
    s1 = (int(s1h[0]) << 64) + int(s1l[0])
    s2 = (int(s2h[0]) << 64) + int(s2l[0])
    return s1, s2, int(n[0]), e[0]


def mean(c) -> float:
    """Sec. V-B mean: (S1 / n) * 2 eps_q, exact rational rounded once to double."""
    s1, _, n, e = sums(c)
    if n == 0:
        raise OracleError(-1, "mean")
    return float(Fraction(s1, n) * 2 * Fraction(float(e)))


def var(c) -> float:
    """Sec. V-B population variance of the dequantized values, from exact sums."""
    s1, s2, n, e = sums(c)
    if n == 0:
        raise OracleError(-1, "var")
    a = 2 * Fraction(float(e))
    return float(a * a * Fraction(n * s2 - s1 * s1, n * n))


def std(c) -> float:
    """Sec. V-B standard deviation: the square root of the population variance
    (the variance rounded once to double, then a correctly rounded square root)."""
    import math

    return math.sqrt(var(c))


def block_means(c) -> np.ndarray:
    """Sec. V-B block-wise means: (S1_b / L_b) * 2 eps_q per block, in FP64."""
    c = _stream(c)
    nb = (header(c)["n"] + 63) // 64
    out = np.zeros(max(nb, 1), np.float64)
    _check(_load().orc_block_means(_ptr(c), c.size, _ptr(out), nb), "block_means")
    return out[:nb].copy()


def cov_sums(a, b):
    """Exact (S_AB, S1_A, S1_B, n) of two streams of one length (Sec. V-D)."""
    a = _stream(a)
    b = _stream(b)
    hi = [np.zeros(1, np.int64) for _ in range(3)]
    lo = [np.zeros(1, np.uint64) for _ in range(3)]
    n = np.zeros(1, np.uint64)
    _check(_load().orc_cov_sums(_ptr(a), a.size, _ptr(b), b.size, _ptr(hi[0]), _ptr(lo[0]),
                                _ptr(hi[1]), _ptr(lo[1]), _ptr(hi[2]), _ptr(lo[2]), _ptr(n)),
           "cov_sums")
    sab, s1a, s1b = ((int(h[0]) << 64) + int(l[0]) for h, l in zip(hi, lo))
    return sab, s1a, s1b, int(n[0])


def cov(a, b) -> float:
    """Sec. V-D population covariance of the dequantized values of two streams,
    2 eps_A 2 eps_B (n S_AB - S1_A S1_B) / n^2 from exact sums, rounded once."""
    sab, s1a, s1b, n = cov_sums(a, b)
    if n == 0:
        raise OracleError(-1, "cov")
    ea = 2 * Fraction(float(header(a)["eps_q"]))
    eb = 2 * Fraction(float(header(b)["eps_q"]))
    return float(ea * eb * Fraction(n * sab - s1a * s1b, n * n))
