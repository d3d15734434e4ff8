"""ctypes binding of libhoszp (see include/hoszp.h for the C ABI)."""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(PKG, "libhoszp.so")

STATUS = {
    0: "OK", -1: "ARG", -2: "CAPACITY", -3: "FORMAT", -4: "MISMATCH", -5: "RANGE",
    -6: "OVERFLOW", -7: "NONFINITE", -8: "TIMEOUT", -9: "CUDA",
}
HEADER_BYTES = 64
EB_MODES = {"abs": 0, "rel": 1}


class HoszpError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"hoszp {what}: {STATUS.get(code, code)} ({code})")
        self.code = code
        self.name = STATUS.get(code, str(code))


_lib = None
_lock = threading.Lock()


class _Request(ctypes.Structure):  # hoszp_request
    _fields_ = [("tag", ctypes.c_uint64), ("op", ctypes.c_int32), ("a", ctypes.c_uint32),
                ("b", ctypes.c_uint32), ("scalar", ctypes.c_double),
                ("arrival_us", ctypes.c_uint64)]


class _Completion(ctypes.Structure):  # hoszp_completion
    _fields_ = [("tag", ctypes.c_uint64), ("op", ctypes.c_int32), ("status", ctypes.c_int32),
                ("value", ctypes.c_double), ("d_out", ctypes.c_void_p),
                ("out_bytes", ctypes.c_uint64), ("arrival_us", ctypes.c_uint64),
                ("start_us", ctypes.c_uint64), ("done_us", ctypes.c_uint64)]


class _ServerStats(ctypes.Structure):  # hoszp_server_stats
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "completed", "pending", "in_flight", "arena_bytes", "arena_in_use",
        "arena_peak", "workspace_bytes", "max_in_flight")]


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libhoszp.so; raises if it has not been built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"libhoszp.so not found at {_LIB_PATH}; build it with "
                "`python -m paper_2408_11971_gb300.build` (needs nvcc, sm_103a)")
        lib = ctypes.CDLL(_LIB_PATH)
        P, U64, SZ, I, D = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int,
                            ctypes.c_double)
        sig = {
            "hoszp_ctx_create": (I, [ctypes.POINTER(P), I]),
            "hoszp_ctx_destroy": (None, [P]),
            "hoszp_ctx_reserve": (I, [P, U64]),
            "hoszp_get_status": (I, [P, ctypes.POINTER(I)]),
            "hoszp_compress_bound": (SZ, [U64]),
            "hoszp_compress": (I, [P, P, U64, P, I, D, I, P, SZ, P, P]),
            "hoszp_decompress": (I, [P, P, SZ, P, U64, P]),
            "hoszp_negate": (I, [P, P, SZ, P, SZ, P, P]),
            "hoszp_add_scalar": (I, [P, P, SZ, D, P, SZ, P, P]),
            "hoszp_sub_scalar": (I, [P, P, SZ, D, P, SZ, P, P]),
            "hoszp_mul_scalar": (I, [P, P, SZ, D, P, SZ, P, P]),
            "hoszp_mul_scalar_exact": (I, [P, P, SZ, D, P, SZ, P, P]),
            "hoszp_add": (I, [P, P, SZ, P, SZ, P, SZ, P, P]),
            "hoszp_sub": (I, [P, P, SZ, P, SZ, P, SZ, P, P]),
            "hoszp_hadamard": (I, [P, P, SZ, P, SZ, P, U64, P, SZ, P, P]),
            "hoszp_mean": (I, [P, P, SZ, P, P]),
            "hoszp_sums": (I, [P, P, SZ, P, P]),
            "hoszp_finish_sums": (I, [P, P, ctypes.c_float, P, P, P]),
            "hoszp_concat": (I, [P, ctypes.c_uint32, P, P, P, I, P, SZ, P, P]),
            "hoszp_selftest_wait": (I, [P, I, U64, P]),
            "hoszp_batch_mul_scalar": (I, [P, D, P, P, P, P]),
            "hoszp_batch_add": (I, [P, P, I, P, P, P, P]),
            "hoszp_batch_compress": (I, [P, ctypes.c_uint32, P, P, P, I, P, P, P, P]),
            "hoszp_var": (I, [P, P, SZ, P, P]),
            "hoszp_std": (I, [P, P, SZ, P, P]),
            "hoszp_cov": (I, [P, P, SZ, P, SZ, P, P]),
            "hoszp_block_means": (I, [P, P, SZ, P, U64, P]),
            "hoszp_batch_create": (I, [P, ctypes.c_uint32, P, P, ctypes.POINTER(P)]),
            "hoszp_batch_destroy": (None, [P]),
            "hoszp_batch_info": (I, [P, P, P]),
            "hoszp_batch_get_status": (I, [P, ctypes.POINTER(I)]),
            "hoszp_batch_mean": (I, [P, P, P]),
            "hoszp_batch_var": (I, [P, P, P]),
            "hoszp_batch_decompress": (I, [P, P, P]),
            "hoszp_batch_negate": (I, [P, P]),
            "hoszp_batch_add_scalar": (I, [P, D, P]),
            "hoszp_batch_tune": (I, [P, P, P, P]),
            "hoszp_batch_config": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I),
                                       ctypes.POINTER(I), ctypes.POINTER(I)]),
            "hoszp_batch_shapes": (I, [P, I]),
            "hoszp_batch_set_shape": (I, [P, I, I]),
            "hoszp_server_create": (I, [I, ctypes.c_uint32, U64, U64, ctypes.c_uint32,
                                        ctypes.POINTER(P)]),
            "hoszp_server_destroy": (None, [P]),
            "hoszp_server_register": (I, [P, P, SZ, ctypes.POINTER(ctypes.c_uint32)]),
            "hoszp_server_submit": (I, [P, ctypes.POINTER(_Request)]),
            "hoszp_server_poll": (I, [P, ctypes.POINTER(_Completion), ctypes.c_uint32,
                                      ctypes.POINTER(ctypes.c_uint32), U64]),
            "hoszp_server_release": (I, [P, P]),
            "hoszp_server_now_us": (U64, [P]),
            "hoszp_server_get_stats": (I, [P, ctypes.POINTER(_ServerStats)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _torch():
    import torch

    return torch


class Context:
    """Owns a hoszp_ctx (device status word + workspace) on one CUDA device.
    One context serves one stream at a time."""

    def __init__(self, device: int = 0):
        lib = load_library()
        self.device = int(device)
        h = ctypes.c_void_p()
        rc = lib.hoszp_ctx_create(ctypes.byref(h), self.device)
        if rc != 0:
            raise HoszpError(rc, "ctx_create")
        self.handle = h
        self._lib = lib

    def close(self):
        if getattr(self, "handle", None):
            self._lib.hoszp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, n: int):
        _check(self._lib.hoszp_ctx_reserve(self.handle, int(n)), "ctx_reserve")

    def status(self) -> int:
        st = ctypes.c_int(0)
        _check(self._lib.hoszp_get_status(self.handle, ctypes.byref(st)), "get_status")
        return st.value

    def check(self, what: str = "device"):
        st = self.status()
        if st != 0:
            raise HoszpError(st, what)


_contexts: dict = {}


def default_context(device: int | None = None) -> Context:
    torch = _torch()
    if device is None:
        device = torch.cuda.current_device()
    ctx = _contexts.get(device)
    if ctx is None:
        ctx = _contexts[device] = Context(device)
    return ctx


def _check(rc: int, what: str):
    if rc != 0:
        raise HoszpError(rc, what)


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream_tensor(c):
    torch = _torch()
    if not isinstance(c, torch.Tensor) or not c.is_cuda or c.dtype != torch.uint8:
        raise TypeError("a compressed stream is a CUDA uint8 tensor")
    return c.contiguous()


def _ctx(ctx, t):
    return ctx if ctx is not None else default_context(t.device.index)


def _finish(ctx, out, size_t, sync, check, what):
    if not sync:
        return out, size_t
    if check:
        ctx.check(what)
    n = int(size_t.item())
    return out[:n]


def compress_bound(n: int) -> int:
    return int(load_library().hoszp_compress_bound(int(n)))


def header(c) -> dict:
    """Header fields of a stream (reads 64 bytes to the host)."""
    import numpy as np

    h = c[:HEADER_BYTES].cpu().numpy().tobytes()
    return dict(
        magic=int.from_bytes(h[0:4], "little"), ndims=h[7],
        dims=[int.from_bytes(h[8 + 4 * i:12 + 4 * i], "little") for i in range(3)],
        eps_q=float(np.frombuffer(h[20:24], np.float32)[0]),
        n=int.from_bytes(h[24:32], "little"), eps=float(np.frombuffer(h[32:40], np.float64)[0]),
        nnc=int.from_bytes(h[40:48], "little"), R=int.from_bytes(h[48:56], "little"),
        qbound=int.from_bytes(h[56:60], "little"))


def compress(x, eb: float, mode: str = "abs", dims=None, out=None, out_bytes=None, stream=None,
             ctx: Context | None = None, sync: bool = True, check: bool = True):
    """Compress a float32 CUDA tensor (Sec. IV-A). Returns the stream as a uint8
    tensor (sync=True) or (buffer, size tensor) without synchronizing."""
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32:
        raise TypeError("compress expects a CUDA float32 tensor")
    x = x.contiguous()
    ctx = _ctx(ctx, x)
    shape = tuple(x.shape) if dims is None else tuple(dims)
    if len(shape) == 0:
        shape = (1,)
    if len(shape) > 3:
        shape = (x.numel(),)
    d3 = (ctypes.c_uint32 * 3)(*(list(shape) + [0] * (3 - len(shape))))
    n = x.numel()
    cap = compress_bound(n)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    if out_bytes is None:
        out_bytes = torch.zeros(1, dtype=torch.int64, device=x.device)
    rc = load_library().hoszp_compress(ctx.handle, _dev_ptr(x), n, d3, len(shape), float(eb),
                                       EB_MODES[mode], _dev_ptr(out), out.numel(),
                                       _dev_ptr(out_bytes), _stream_ptr(stream))
    _check(rc, "compress")
    return _finish(ctx, out, out_bytes, sync, check, "compress")


def decompress(c, n: int | None = None, out=None, stream=None, ctx: Context | None = None,
               check: bool = True):
    torch = _torch()
    c = _stream_tensor(c)
    ctx = _ctx(ctx, c)
    if n is None:
        n = header(c)["n"]
    if out is None:
        out = torch.empty(max(int(n), 0), dtype=torch.float32, device=c.device)
    rc = load_library().hoszp_decompress(ctx.handle, _dev_ptr(c), c.numel(), _dev_ptr(out), int(n),
                                         _stream_ptr(stream))
    _check(rc, "decompress")
    if check:
        ctx.check("decompress")
    return out


def _unary(fn, what, c, extra, out, out_bytes, inplace, stream, ctx, sync, check):
    torch = _torch()
    c = _stream_tensor(c)
    ctx = _ctx(ctx, c)
    if inplace:
        out = c
    elif out is None:
        grows = what in ("mul_scalar", "mul_scalar_exact")  # outputs that can outgrow the input
        out = torch.empty(max(c.numel(), compress_bound(header(c)["n"])) if grows else c.numel(),
                          dtype=torch.uint8, device=c.device)
    if out_bytes is None:
        out_bytes = torch.zeros(1, dtype=torch.int64, device=c.device)
    rc = fn(ctx.handle, _dev_ptr(c), c.numel(), *extra, _dev_ptr(out), out.numel(),
            _dev_ptr(out_bytes), _stream_ptr(stream))
    _check(rc, what)
    return _finish(ctx, out, out_bytes, sync, check, what)


def negate(c, out=None, out_bytes=None, inplace: bool = False, stream=None, ctx=None,
           sync: bool = True, check: bool = True):
    """Negation in fully compressed space (Sec. V-A)."""
    return _unary(load_library().hoszp_negate, "negate", c, (), out, out_bytes, inplace, stream,
                  ctx, sync, check)


def add_scalar(c, s: float, out=None, out_bytes=None, inplace: bool = False, stream=None,
               ctx=None, sync: bool = True, check: bool = True):
    """Scalar addition in fully compressed space (Sec. V-A)."""
    return _unary(load_library().hoszp_add_scalar, "add_scalar", c, (ctypes.c_double(s),), out,
                  out_bytes, inplace, stream, ctx, sync, check)


def sub_scalar(c, s: float, out=None, out_bytes=None, inplace: bool = False, stream=None,
               ctx=None, sync: bool = True, check: bool = True):
    """Scalar subtraction in fully compressed space (Sec. V-A): O' = O - rho_s."""
    return _unary(load_library().hoszp_sub_scalar, "sub_scalar", c, (ctypes.c_double(s),), out,
                  out_bytes, inplace, stream, ctx, sync, check)


def mul_scalar(c, s: float, out=None, out_bytes=None, stream=None, ctx=None, sync: bool = True,
               check: bool = True):
    """Scalar multiplication through the quantized integers (Sec. V-A)."""
    return _unary(load_library().hoszp_mul_scalar, "mul_scalar", c, (ctypes.c_double(s),), out,
                  out_bytes, False, stream, ctx, sync, check)


def mul_scalar_exact(c, s: float, out=None, out_bytes=None, stream=None, ctx=None,
                     sync: bool = True, check: bool = True):
    """Multiplication by the scalar itself, q' = floor(q s + 1/2), through the
    quantized integers."""
    return _unary(load_library().hoszp_mul_scalar_exact, "mul_scalar_exact", c,
                  (ctypes.c_double(s),), out, out_bytes, False, stream, ctx, sync, check)


def _bivariate(fn, what, a, b, out, out_bytes, stream, ctx, sync, check):
    torch = _torch()
    a = _stream_tensor(a)
    b = _stream_tensor(b)
    ctx = _ctx(ctx, a)
    if out is None:
        out = torch.empty(compress_bound(header(a)["n"]), dtype=torch.uint8, device=a.device)
    if out_bytes is None:
        out_bytes = torch.zeros(1, dtype=torch.int64, device=a.device)
    rc = fn(ctx.handle, _dev_ptr(a), a.numel(), _dev_ptr(b), b.numel(), _dev_ptr(out),
            out.numel(), _dev_ptr(out_bytes), _stream_ptr(stream))
    _check(rc, what)
    return _finish(ctx, out, out_bytes, sync, check, what)


def concat(streams, dims, out=None, out_bytes=None, stream=None, ctx=None, sync: bool = True,
           check: bool = True):
    """The streams of consecutive shards of one field (every shard but the last of
    whole blocks, one bound) joined into the field's stream of shape dims
    (hoszp_concat; Sec. VI-B5)."""
    torch = _torch()
    ss = [_stream_tensor(c) for c in streams]
    if not ss:
        raise ValueError("no streams")
    ctx = _ctx(ctx, ss[0])
    n = 1
    for d in dims:
        n *= int(d)
    if out is None:
        out = torch.empty(compress_bound(n), dtype=torch.uint8, device=ss[0].device)
    if out_bytes is None:
        out_bytes = torch.zeros(1, dtype=torch.int64, device=ss[0].device)
    k = len(ss)
    ptrs = (ctypes.c_void_p * k)(*[_dev_ptr(c) for c in ss])
    sizes = (ctypes.c_size_t * k)(*[c.numel() for c in ss])
    d3 = (ctypes.c_uint32 * 3)(*(list(dims) + [0, 0, 0])[:3])
    rc = load_library().hoszp_concat(ctx.handle, k, ptrs, sizes, d3, len(dims), _dev_ptr(out),
                                     out.numel(), _dev_ptr(out_bytes), _stream_ptr(stream))
    _check(rc, "concat")
    return _finish(ctx, out, out_bytes, sync, check, "concat")


def add(a, b, out=None, out_bytes=None, stream=None, ctx=None, sync: bool = True,
        check: bool = True):
    """Element-wise addition of two streams (Sec. V-C)."""
    return _bivariate(load_library().hoszp_add, "add", a, b, out, out_bytes, stream, ctx, sync,
                      check)


def sub(a, b, out=None, out_bytes=None, stream=None, ctx=None, sync: bool = True,
        check: bool = True):
    """Element-wise subtraction A - B of two streams (Sec. V-C)."""
    return _bivariate(load_library().hoszp_sub, "sub", a, b, out, out_bytes, stream, ctx, sync,
                      check)


def hadamard(a, b, out=None, out_bytes=None, scratch=None, stream=None, ctx=None,
             sync: bool = True, check: bool = True):
    """Hadamard product of two streams (Sec. V-C), q' = floor(2 eps q_A q_B + 1/2).
    `scratch`: an int32 CUDA tensor of n values (allocated when not given)."""
    torch = _torch()
    a = _stream_tensor(a)
    b = _stream_tensor(b)
    ctx = _ctx(ctx, a)
    n = header(a)["n"]
    if scratch is None:
        scratch = torch.empty(max(n, 4), dtype=torch.int32, device=a.device)
    if out is None:
        out = torch.empty(compress_bound(n), dtype=torch.uint8, device=a.device)
    if out_bytes is None:
        out_bytes = torch.zeros(1, dtype=torch.int64, device=a.device)
    rc = load_library().hoszp_hadamard(ctx.handle, _dev_ptr(a), a.numel(), _dev_ptr(b), b.numel(),
                                       _dev_ptr(scratch), n, _dev_ptr(out), out.numel(),
                                       _dev_ptr(out_bytes), _stream_ptr(stream))
    _check(rc, "hadamard")
    return _finish(ctx, out, out_bytes, sync, check, "hadamard")


def _moment(fn, what, c, out, stream, ctx, sync, check):
    torch = _torch()
    c = _stream_tensor(c)
    ctx = _ctx(ctx, c)
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=c.device)
    rc = fn(ctx.handle, _dev_ptr(c), c.numel(), _dev_ptr(out), _stream_ptr(stream))
    _check(rc, what)
    if not sync:
        return out
    if check:
        ctx.check(what)
    return float(out.item())


def sums(c, stream=None, ctx=None):
    """The stream's exact sums as the five words of hoszp_sums (S1 low/high,
    S2 low/high, n), read back to the host."""
    torch = _torch()
    c = _stream_tensor(c)
    ctx = _ctx(ctx, c)
    w = torch.zeros(5, dtype=torch.int64, device=c.device)
    _check(load_library().hoszp_sums(ctx.handle, _dev_ptr(c), c.numel(), _dev_ptr(w),
                                     _stream_ptr(stream)), "sums")
    ctx.check("sums")
    return [int(v) & ((1 << 64) - 1) for v in w.cpu().tolist()]


def finish_sums(words, eps_q, device=0, stream=None, ctx=None):
    """(mean, population variance) of a field from the five words of its exact
    sums combined over shards (hoszp_finish_sums: the kernels' FP64 finish)."""
    torch = _torch()
    w = torch.tensor([int(v) - (1 << 64) if int(v) >> 63 else int(v) for v in words],
                     dtype=torch.int64, device=torch.device("cuda", device))
    if ctx is None:
        ctx = _ctx(None, w)
    out = torch.zeros(2, dtype=torch.float64, device=w.device)
    _check(load_library().hoszp_finish_sums(ctx.handle, _dev_ptr(w), ctypes.c_float(eps_q),
                                            _dev_ptr(out), ctypes.c_void_p(out.data_ptr() + 8),
                                            _stream_ptr(stream)), "finish_sums")
    ctx.check("finish_sums")
    m, v = out.cpu().tolist()
    return m, v


def mean(c, out=None, stream=None, ctx=None, sync: bool = True, check: bool = True):
    """Mean from the quantized integers (Sec. V-B)."""
    return _moment(load_library().hoszp_mean, "mean", c, out, stream, ctx, sync, check)


def var(c, out=None, stream=None, ctx=None, sync: bool = True, check: bool = True):
    """Population variance from exact integer sums (Sec. V-B)."""
    return _moment(load_library().hoszp_var, "var", c, out, stream, ctx, sync, check)


def std(c, out=None, stream=None, ctx=None, sync: bool = True, check: bool = True):
    """Standard deviation: square root of the population variance (Sec. V-B)."""
    return _moment(load_library().hoszp_std, "std", c, out, stream, ctx, sync, check)


def cov(a, b, out=None, stream=None, ctx=None, sync: bool = True, check: bool = True):
    """Population covariance of two streams of one length (their bounds may
    differ), from exact integer sums in one pass (Sec. V-D)."""
    torch = _torch()
    a = _stream_tensor(a)
    b = _stream_tensor(b)
    ctx = _ctx(ctx, a)
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=a.device)
    _check(load_library().hoszp_cov(ctx.handle, _dev_ptr(a), a.numel(), _dev_ptr(b), b.numel(),
                                    _dev_ptr(out), _stream_ptr(stream)), "cov")
    if not sync:
        return out
    if check:
        ctx.check("cov")
    return float(out.item())


def block_means(c, out=None, stream=None, ctx=None, sync: bool = True, check: bool = True):
    """Block-wise means (Sec. V-B): a float64 CUDA tensor with one mean per
    64-value block, (S1_b / L_b) * 2 eps_q."""
    torch = _torch()
    c = _stream_tensor(c)
    ctx = _ctx(ctx, c)
    nb = (header(c)["n"] + 63) // 64
    if out is None:
        out = torch.empty(max(nb, 1), dtype=torch.float64, device=c.device)
    _check(load_library().hoszp_block_means(ctx.handle, _dev_ptr(c), c.numel(), _dev_ptr(out), nb,
                                            _stream_ptr(stream)), "block_means")
    if sync and check:
        ctx.check("block_means")
    return out[:nb]


# ---------------------------------------------------------------- traditional workflow (float ops)
def _fop_lib():
    lib = load_library()
    if not getattr(lib, "_fop_ready", False):
        P, U64, F, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_float, ctypes.c_int
        lib.hoszp_fop_axpb.restype = I
        lib.hoszp_fop_axpb.argtypes = [P, P, U64, F, F, P]
        lib.hoszp_fop_add.restype = I
        lib.hoszp_fop_add.argtypes = [P, P, P, U64, P]
        lib.hoszp_fop_moments.restype = I
        lib.hoszp_fop_moments.argtypes = [P, P, U64, I, P, P]
        lib._fop_ready = True
    return lib


def fop_axpb(x, a: float, b: float, out=None, stream=None):
    """y = a x + b on a float32 CUDA tensor (traditional-workflow operator)."""
    torch = _torch()
    out = torch.empty_like(x) if out is None else out
    _check(_fop_lib().hoszp_fop_axpb(_dev_ptr(x), _dev_ptr(out), x.numel(), a, b,
                                     _stream_ptr(stream)), "fop_axpb")
    return out


def fop_add(x, y, out=None, stream=None):
    torch = _torch()
    out = torch.empty_like(x) if out is None else out
    _check(_fop_lib().hoszp_fop_add(_dev_ptr(x), _dev_ptr(y), _dev_ptr(out), x.numel(),
                                    _stream_ptr(stream)), "fop_add")
    return out


def fop_moments(x, variance: bool, out=None, stream=None, ctx=None):
    torch = _torch()
    ctx = _ctx(ctx, x)
    out = torch.zeros(1, dtype=torch.float64, device=x.device) if out is None else out
    _check(_fop_lib().hoszp_fop_moments(ctx.handle, _dev_ptr(x), x.numel(), 1 if variance else 0,
                                        _dev_ptr(out), _stream_ptr(stream)), "fop_moments")
    return out


class Batch:
    """A batch plan over resident streams (one snapshot's fields): one launch
    per operator over all of them. Keeps references to the stream tensors,
    which the plan reads (and, for negate / add_scalar, modifies) in place."""

    def __init__(self, streams, ctx=None):
        torch = _torch()
        self._streams = [_stream_tensor(c) for c in streams]
        if not self._streams:
            raise ValueError("empty batch")
        self.ctx = _ctx(ctx, self._streams[0])
        self._lib = load_library()
        nf = len(self._streams)
        ptrs = (ctypes.c_void_p * nf)(*[c.data_ptr() for c in self._streams])
        sizes = (ctypes.c_size_t * nf)(*[c.numel() for c in self._streams])
        h = ctypes.c_void_p()
        torch.cuda.synchronize(self._streams[0].device)
        _check(self._lib.hoszp_batch_create(self.ctx.handle, nf, ptrs, sizes, ctypes.byref(h)),
               "batch_create")
        self.handle = h
        self.nfields = nf
        self.device = self._streams[0].device

    def close(self):
        if getattr(self, "handle", None):
            self._lib.hoszp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self) -> int:
        st = ctypes.c_int(0)
        _check(self._lib.hoszp_batch_get_status(self.handle, ctypes.byref(st)),
               "batch_get_status")
        return st.value

    def check(self, what: str = "batch"):
        st = self.status()
        if st != 0:
            raise HoszpError(st, what)

    def _moment(self, fn, what, out, stream, sync, check):
        torch = _torch()
        if out is None:
            out = torch.empty(self.nfields, dtype=torch.float64, device=self.device)
        _check(fn(self.handle, _dev_ptr(out), _stream_ptr(stream)), what)
        if sync:
            torch.cuda.synchronize(self.device)
            if check:
                self.check(what)
        return out

    def mean(self, out=None, stream=None, sync: bool = True, check: bool = True):
        """Per-field means (Sec. V-B), one launch."""
        return self._moment(self._lib.hoszp_batch_mean, "batch_mean", out, stream, sync, check)

    def var(self, out=None, stream=None, sync: bool = True, check: bool = True):
        """Per-field population variances (Sec. V-B), one launch."""
        return self._moment(self._lib.hoszp_batch_var, "batch_var", out, stream, sync, check)

    def decompress(self, outs=None, stream=None, sync: bool = True, check: bool = True):
        """Every field decompressed (Fig. 2), one launch: a list of float32 CUDA
        tensors (allocated when not given, n_f values each)."""
        torch = _torch()
        if outs is None:
            outs = [torch.empty(header(c)["n"], dtype=torch.float32, device=self.device)
                    for c in self._streams]
        ptrs = torch.tensor([o.data_ptr() for o in outs], dtype=torch.int64, device=self.device)
        _check(self._lib.hoszp_batch_decompress(self.handle, _dev_ptr(ptrs), _stream_ptr(stream)),
               "batch_decompress")
        self._ptrs = ptrs  # kept alive until the next call (the launch reads it)
        if sync:
            torch.cuda.synchronize(self.device)
            if check:
                self.check("batch_decompress")
        return outs

    def negate(self, stream=None):
        """Every field negated in place (Sec. V-A), one launch."""
        _check(self._lib.hoszp_batch_negate(self.handle, _stream_ptr(stream)), "batch_negate")

    def add_scalar(self, s: float, stream=None):
        """s added to every field in place (Sec. V-A), one launch (+ a per-field
        quantization of s)."""
        _check(self._lib.hoszp_batch_add_scalar(self.handle, float(s), _stream_ptr(stream)),
               "batch_add_scalar")

    def _outputs(self, outs, bound_n):
        torch = _torch()
        if outs is None:
            outs = [torch.empty(bound_n(c), dtype=torch.uint8, device=self.device)
                    for c in self._streams]
        ptrs = torch.tensor([o.data_ptr() for o in outs], dtype=torch.int64, device=self.device)
        caps = torch.tensor([o.numel() for o in outs], dtype=torch.int64, device=self.device)
        sizes = torch.zeros(len(outs), dtype=torch.int64, device=self.device)
        return outs, ptrs, caps, sizes

    def _produced(self, what, outs, ptrs, caps, sizes, sync, check):
        self._keep = (ptrs, caps)  # kept alive until the next call (the launches read them)
        if not sync:
            return outs, sizes
        _torch().cuda.synchronize(self.device)
        if check:
            self.check(what)
        return [o[: int(k)] for o, k in zip(outs, sizes.cpu().tolist())]

    def mul_scalar(self, s: float, outs=None, stream=None, sync: bool = True,
                   check: bool = True):
        """Every field times s (Sec. V-A), one launch over all fields (+ one
        scan and one placement launch): a list of output streams."""
        outs, ptrs, caps, sizes = self._outputs(outs, lambda c: compress_bound(header(c)["n"]))
        _check(self._lib.hoszp_batch_mul_scalar(self.handle, float(s), _dev_ptr(ptrs),
                                                _dev_ptr(caps), _dev_ptr(sizes),
                                                _stream_ptr(stream)), "batch_mul_scalar")
        return self._produced("batch_mul_scalar", outs, ptrs, caps, sizes, sync, check)

    def add(self, other: "Batch", subtract: bool = False, outs=None, stream=None,
            sync: bool = True, check: bool = True):
        """Field by field A_f + B_f (or A_f - B_f; Sec. V-C) of this plan and
        another with the same fields' shapes and bounds, one launch."""
        outs, ptrs, caps, sizes = self._outputs(outs, lambda c: compress_bound(header(c)["n"]))
        _check(self._lib.hoszp_batch_add(self.handle, other.handle, 1 if subtract else 0,
                                         _dev_ptr(ptrs), _dev_ptr(caps), _dev_ptr(sizes),
                                         _stream_ptr(stream)), "batch_add")
        return self._produced("batch_add", outs, ptrs, caps, sizes, sync, check)

    OPS = ("mean", "var", "decompress")

    def tune(self, outs=None, stream=None):
        """Pick each operator's launch shape from timed runs on the plan's data
        (decompression too when outs, one float32 tensor per field, is given);
        returns the picks."""
        torch = _torch()
        res = torch.empty(self.nfields, dtype=torch.float64, device=self.device)
        ptrs = None
        if outs is not None:
            ptrs = torch.tensor([o.data_ptr() for o in outs], dtype=torch.int64, device=self.device)
        _check(self._lib.hoszp_batch_tune(self.handle, _dev_ptr(res),
                                          _dev_ptr(ptrs) if ptrs is not None else None,
                                          _stream_ptr(stream)), "batch_tune")
        self.check("batch_tune")
        return {op: self.config(i) for i, op in enumerate(self.OPS)}

    def config(self, op: int):
        st, cps, wpg, pg = (ctypes.c_int(0) for _ in range(4))
        _check(self._lib.hoszp_batch_config(self.handle, int(op), ctypes.byref(st),
                                            ctypes.byref(cps), ctypes.byref(wpg),
                                            ctypes.byref(pg)), "batch_config")
        return {"stages": st.value, "ctas_per_sm": cps.value, "warps_per_group": wpg.value,
                "plane_groups": pg.value}

    def shapes(self, op: int) -> int:
        """Number of launch shapes the tuner tries for op (0 mean, 1 var, 2 decompress)."""
        n = self._lib.hoszp_batch_shapes(self.handle, int(op))
        if n < 0:
            raise HoszpError(n, "batch_shapes")
        return n

    def set_shape(self, op: int, index: int):
        """Select launch shape `index` of op without timing."""
        _check(self._lib.hoszp_batch_set_shape(self.handle, int(op), int(index)), "batch_set_shape")


def batch_compress(xs, eb, mode: str = "rel", outs=None, stream=None, ctx=None,
                   sync: bool = True, check: bool = True):
    """Many float32 fields (1-D CUDA tensors) compressed in one launch over all
    their tiles (+ a range pass for relative bounds, one scan and one placement
    launch); eb: one bound per field (or one for all). Returns the streams."""
    torch = _torch()
    xs = [x.contiguous() for x in xs]
    if not xs:
        raise ValueError("no fields")
    dev = xs[0].device
    ctx = _ctx(ctx, xs[0])
    k = len(xs)
    ebs = list(eb) if hasattr(eb, "__len__") else [float(eb)] * k
    if outs is None:
        outs = [torch.empty(compress_bound(x.numel()), dtype=torch.uint8, device=dev) for x in xs]
    sizes = torch.zeros(k, dtype=torch.int64, device=dev)
    P = ctypes.c_void_p
    xp = (P * k)(*[x.data_ptr() for x in xs])
    ns = (ctypes.c_uint64 * k)(*[x.numel() for x in xs])
    es = (ctypes.c_double * k)(*[float(e) for e in ebs])
    op = (P * k)(*[o.data_ptr() for o in outs])
    cp = (ctypes.c_size_t * k)(*[o.numel() for o in outs])
    rc = load_library().hoszp_batch_compress(ctx.handle, k, xp, ns, es,
                                             1 if mode == "rel" else 0, op, cp, _dev_ptr(sizes),
                                             _stream_ptr(stream))
    _check(rc, "batch_compress")
    if not sync:
        return outs, sizes
    torch.cuda.synchronize(dev)
    if check:
        ctx.check("batch_compress")
    return [o[: int(n)] for o, n in zip(outs, sizes.cpu().tolist())]


class _DevBuf:
    """A device buffer exposed through the CUDA array interface (no copy)."""

    def __init__(self, ptr: int, nbytes: int, typestr: str, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


class Server:
    """Continuous-batching server over resident streams (hoszp_server_*).

    register() the resident streams, submit() requests (optionally with an
    arrival time on the server's clock), poll() completions. An output stays
    in the server's arena until release(); output() views it as a tensor."""

    OPS = {"mean": 0, "var": 1, "negate": 2, "add_scalar": 3, "mul_scalar": 4, "add": 5,
           "sub": 6, "decompress": 7}
    OP_NAMES = {v: k for k, v in OPS.items()}

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int = 8 << 30,
                 max_n: int = 1 << 27, sms_per_request: int = 0):
        self._lib = load_library()
        self.device = int(device)
        h = ctypes.c_void_p()
        _check(self._lib.hoszp_server_create(self.device, int(slots), int(hbm_budget), int(max_n),
                                             int(sms_per_request), ctypes.byref(h)),
               "server_create")
        self.handle = h
        self._streams = []

    def close(self):
        if getattr(self, "handle", None):
            self._lib.hoszp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, c) -> int:
        c = _stream_tensor(c)
        _torch().cuda.synchronize(c.device)
        sid = ctypes.c_uint32(0)
        _check(self._lib.hoszp_server_register(self.handle, _dev_ptr(c), c.numel(),
                                               ctypes.byref(sid)), "server_register")
        self._streams.append(c)  # keeps the stream alive while the server may read it
        return sid.value

    def submit(self, op, a: int, b: int = 0, scalar: float = 0.0, tag: int = 0,
               arrival_us: int = 0):
        r = _Request(int(tag), self.OPS[op] if isinstance(op, str) else int(op), int(a), int(b),
                     float(scalar), int(arrival_us))
        _check(self._lib.hoszp_server_submit(self.handle, ctypes.byref(r)), "server_submit")

    def poll(self, max_n: int = 256, wait_us: int = 0):
        buf = (_Completion * max_n)()
        n = ctypes.c_uint32(0)
        _check(self._lib.hoszp_server_poll(self.handle, buf, max_n, ctypes.byref(n), int(wait_us)),
               "server_poll")
        return [{k: getattr(buf[i], k) for k, _ in _Completion._fields_} for i in range(n.value)]

    def output(self, comp):
        """The completion's output as a CUDA tensor view (uint8 stream or float32 values)."""
        torch = _torch()
        if not comp["d_out"]:
            return None
        if comp["op"] == self.OPS["decompress"]:
            v = _DevBuf(comp["d_out"], comp["out_bytes"], "<f4", comp["out_bytes"] // 4)
        else:
            v = _DevBuf(comp["d_out"], comp["out_bytes"], "|u1", comp["out_bytes"])
        return torch.as_tensor(v, device=torch.device("cuda", self.device))

    def release(self, comp_or_ptr):
        ptr = comp_or_ptr["d_out"] if isinstance(comp_or_ptr, dict) else comp_or_ptr
        if ptr:
            _check(self._lib.hoszp_server_release(self.handle, ctypes.c_void_p(ptr)),
                   "server_release")

    def now_us(self) -> int:
        return int(self._lib.hoszp_server_now_us(self.handle))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(self._lib.hoszp_server_get_stats(self.handle, ctypes.byref(st)), "server_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}
